"""Plain FP64 reference of the surrogate MLP -- TEST INFRASTRUCTURE ONLY.

Network: n_in -> H -> H -> n_out, GELU(x) = x/2 (1 + erf(x/sqrt 2)) after the
two hidden layers; loss = mean over batch x n_out of (y_hat - t_hat)^2 with
t_hat = (t - shift) / scale.  Backward by the chain rule, AdamW by its
published update (Loshchilov & Hutter, decoupled weight decay).

With emulate=True the GEMM operands are rounded to bfloat16 (round to
nearest even) at the points where the tensor-core kernels round them, so
that both sides take those rounding decisions on the same inputs; every
other operation is FP64.  Flat parameter layout: W1, b1, W2, b2, W3, b3 with
W row-major [out][in].
"""
import numpy as np
from scipy.special import erf


def bf16(x):
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def dgelu(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def unflatten(flat, n_in, n_hid, n_out):
    dims = [n_in, n_hid, n_hid, n_out]
    out, off = [], 0
    for l in range(3):
        i, o = dims[l], dims[l + 1]
        W = np.asarray(flat[off:off + o * i], dtype=np.float64).reshape(o, i)
        off += o * i
        b = np.asarray(flat[off:off + o], dtype=np.float64)
        off += o
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(layers, X, emulate=True):
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    A = r(X)
    cache = {"A": [A], "Z": []}
    for l, (W, b) in enumerate(layers):
        Z = A @ r(W).T + b
        cache["Z"].append(Z)
        if l < 2:
            A = r(gelu(Z))
            cache["A"].append(A)
    return cache["Z"][-1], cache


def loss_and_grads(layers, X, T, scale, shift, emulate=True):
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    Yh, cache = forward(layers, X, emulate)
    That = (T - shift) / scale
    B, n_out = Yh.shape
    R = Yh - That
    loss = np.mean(R * R)
    dZ = 2.0 * R / (B * n_out)
    grads = [None] * 3
    for l in (2, 1, 0):
        W, _ = layers[l]
        A = cache["A"][l]
        grads[l] = (r(dZ).T @ A, dZ.sum(axis=0))
        if l > 0:
            dZ = (r(dZ) @ r(W)) * dgelu(cache["Z"][l - 1])
    return loss, grads


def adamw(p, g, m, v, t, lr, b1, b2, eps, wd):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * (mh / (np.sqrt(vh) + eps) + wd * p), m, v

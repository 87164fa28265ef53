"""Surrogate MLP kernels (tcgen05 BF16 GEMMs, FP32 accumulation) against the
FP64 oracle MLP with the same BF16 rounding points.

Tolerance, element by element: |got - want| <= C * 2^-8 * (|want| + max|want|)
over each output or gradient block, with C = 1/2.  Both sides round the GEMM
operands to bfloat16 (unit roundoff 2^-8) at the same points; what remains is
FP32 accumulation order and FP32 GELU against FP64 (about 1e-6 relative to
the terms) and the rare bfloat16 rounding decision that flips on a last-bit
difference, which moves one operand by at most 2^-8 of itself.  A
mis-addressed row or column, a wrong bias lane or a dropped term moves an
element by the size of the terms, far beyond this bound.  Each check also
reports the worst element and how many exceed the tighter 2^-12 bound.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


C_BF16 = 0.5


def _check(got, want, what, c=C_BF16):
    """Element-wise bound scaled by bfloat16 precision (module docstring)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    scale = np.abs(want) + np.max(np.abs(want))
    err = np.abs(got - want)
    ratio = err / (2.0 ** -8 * scale + 1e-300)
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    tight = int(np.sum(err > 2.0 ** -12 * scale))
    print(f"{what}: worst |err| = {ratio[worst]:.3f} x 2^-8 (|want|+max|want|) at {worst} "
          f"(got {got[worst]:.6e}, want {want[worst]:.6e}); {tight} of {err.size} beyond 2^-12")
    assert ratio[worst] <= c, f"{what}: element {worst} off by {ratio[worst]:.3f} x 2^-8 scale"


def _setup(n_in, n_hid, n_out, B, seed):
    import paper_2609_14831_b300 as cg
    rng = np.random.default_rng(seed)
    m = cg.MLP(n_in, n_hid, n_out, seed=seed, device=0)
    layers = [(rng.normal(size=(n_hid, n_in)) / np.sqrt(n_in), rng.normal(size=n_hid) * 0.1),
              (rng.normal(size=(n_hid, n_hid)) / np.sqrt(n_hid), rng.normal(size=n_hid) * 0.1),
              (rng.normal(size=(n_out, n_hid)) / np.sqrt(n_hid), rng.normal(size=n_out) * 0.1)]
    flat = omlp.flatten(layers).astype(np.float32)
    m.set_params(flat)
    layers32 = omlp.unflatten(flat.astype(np.float64), n_in, n_hid, n_out)
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    T = rng.normal(size=(B, n_out)).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, n_out).astype(np.float32)
    shift = rng.normal(size=n_out).astype(np.float32)
    m.set_output_affine(scale, shift)
    return m, layers32, X, T, scale.astype(np.float64), shift.astype(np.float64)


@pytest.mark.parametrize("dims", [(32, 512, 848, 300), (5, 64, 70, 129), (32, 512, 848, 1024)])
def test_mlp_forward_matches_oracle(dims):
    n_in, n_hid, n_out, B = dims
    m, layers, X, T, scale, shift = _setup(n_in, n_hid, n_out, B, seed=41)
    y = m.forward(X).cpu().numpy().astype(np.float64)
    m.status()
    Yh, _ = omlp.forward(layers, X.astype(np.float64), emulate=True)
    want = scale * Yh + shift
    assert y.shape == (B, n_out)
    _check(y, want, f"forward {dims}")


@pytest.mark.parametrize("dims", [(32, 512, 848, 300), (5, 64, 70, 129)])
def test_mlp_gradients_match_oracle(dims):
    n_in, n_hid, n_out, B = dims
    m, layers, X, T, scale, shift = _setup(n_in, n_hid, n_out, B, seed=42)
    loss = m.backward(X, T).cpu().numpy()[0]
    m.status()
    want_loss, grads = omlp.loss_and_grads(layers, X.astype(np.float64), T.astype(np.float64), scale, shift,
                                           emulate=True)
    assert abs(loss - want_loss) <= 5e-3 * abs(want_loss)
    got = omlp.unflatten(m.params(grads=True).astype(np.float64), n_in, n_hid, n_out)
    for l in range(3):
        _check(got[l][0], grads[l][0], f"dW{l + 1} {dims}")
        _check(got[l][1], grads[l][1], f"db{l + 1} {dims}")


def test_adamw_step_matches_published_update():
    m, layers, X, T, scale, shift = _setup(6, 64, 10, 128, seed=43)
    p0 = m.params().astype(np.float64)
    m.backward(X, T)
    g = m.params(grads=True).astype(np.float64)
    m.step(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8, weight_decay=0.01)
    m.status()
    p1 = m.params().astype(np.float64)
    # decoupled weight decay on weights only
    nl = omlp.unflatten(np.arange(p0.size), 6, 64, 10)
    is_w = np.zeros(p0.size, dtype=bool)
    for W, _ in nl:
        is_w[W.ravel().astype(int)] = True
    want = np.empty_like(p0)
    for mask, wd in ((is_w, 0.01), (~is_w, 0.0)):
        want[mask], _, _ = omlp.adamw(p0[mask], g[mask], 0.0, 0.0, 1, 1e-2, 0.9, 0.99, 1e-8, wd)
    np.testing.assert_allclose(p1, want, rtol=1e-5, atol=1e-7)


def test_training_reduces_loss():
    import torch
    import paper_2609_14831_b300 as cg
    rng = np.random.default_rng(44)
    m = cg.MLP(8, 128, 16, seed=44, device=0)
    A = rng.normal(size=(8, 16))
    X = rng.uniform(-1, 1, size=(1024, 8)).astype(np.float32)
    Y = np.tanh(X @ A).astype(np.float32)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    losses = []
    for it in range(300):
        losses.append(float(m.backward(Xd, Yd).item()))
        m.step(lr=3e-3)
    m.status()
    assert losses[-1] < 0.05 * losses[0], (losses[0], losses[-1])


def test_linear_skip_term():
    """y = scale * y_hat + shift + J x, with J x in FP32 on the CUDA cores."""
    n_in, n_hid, n_out, B = 32, 512, 848, 200
    m, layers, X, T, scale, shift = _setup(n_in, n_hid, n_out, B, seed=45)
    rng = np.random.default_rng(45)
    J = (rng.normal(size=(n_out, n_in)) * 0.3).astype(np.float32)
    m.set_linear(J)
    y = m.forward(X).cpu().numpy().astype(np.float64)
    Yh, _ = omlp.forward(layers, X.astype(np.float64), emulate=True)
    want = scale * Yh + shift + X.astype(np.float64) @ J.astype(np.float64).T
    _check(y, want, "forward with J x")
    # the loss sees targets with the linear part removed: T = shift + J x
    # (+ scale * network) gives zero residual for the network's own output
    T_exact = (want).astype(np.float32)
    loss = m.backward(X, T_exact).cpu().numpy()[0]
    assert loss < 1e-4
    m.set_linear(None)
    y0 = m.forward(X).cpu().numpy().astype(np.float64)
    _check(y0, scale * Yh + shift, "forward after J removed")


def test_replayed_backward_graph_equals_direct_launches():
    """The second call with the same buffers captures the forward/backward
    pass as a CUDA graph and later calls replay it: the gradients must equal
    the first (direct) call's bit for bit, the loss accumulates into the
    caller's buffer, and a new buffer falls back to direct launches."""
    import torch
    m, layers, X, T, scale, shift = _setup(32, 512, 848, 300, seed=44)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grads = []
    for _ in range(4):                     # direct, capture + replay, replay, replay
        m.backward(Xd, Td, loss=loss)
        grads.append(m.params(grads=True))
    m.status()
    for g in grads[1:]:
        np.testing.assert_array_equal(g, grads[0])
    one = m.backward(Xd, Td).item()        # a new loss buffer: direct launches again
    assert abs(loss.item() - 4 * one) <= 1e-5 * abs(4 * one)
    np.testing.assert_array_equal(m.params(grads=True), grads[0])
    want_loss, _ = omlp.loss_and_grads(layers, X.astype(np.float64), T.astype(np.float64), scale, shift,
                                       emulate=True)
    assert abs(one - want_loss) <= 5e-3 * abs(want_loss)

"""Plain CPU oracle for the projected CUT flow -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the product library: it
evaluates every commutator by direct operator-string multiplication
(oracle/cut_oracle.c) and composes the flow from the paper's definitions:

  * Eq. (block-generator): eta = [H_d, H_od], with H_d the coordinates the
    diagonal mask D selects (Pauli strings over {I, Z}; fermion monomials
    whose creator and annihilator sets coincide) and H_od = H - H_d.
  * Eq. (coflow) + Eq. (projected-flow): dH/ds = P[eta, H],
    dX/ds = P[eta, X], with P applied after the exact, normal-ordered
    commutator (Sec. 2.1).
  * Sec. 2.4 (dual / adjoint traversal): the vector-Jacobian product of the
    right-hand side by the chain rule through the same string algebra.
  * Flow integrators: classical RK4 and Dormand-Prince 5(4) (the paper does
    not name its integrator; the workloads fix RK4 / adaptive RK45).

Coefficient conventions: H = sum_k h_k O_k with real h_k.  The generator is
returned as its complex expansion; real generator coordinates xi follow
eta = i sum xi_g G_g for Pauli strings and eta = sum xi_g G_g for fermions.

Every function here is pinned by tests/test_oracle_*.py against dense
matrices, closed forms and invariants (no test compares it to itself).
"""
import ctypes
import os

import numpy as np

from . import build as _build

ALG_PAULI = 0
ALG_FERMION = 1
ALG_PAULI_BOSON = 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        for name in ("oracle_product", "oracle_commutator"):
            fn = getattr(lib, name)
            fn.restype = vp
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp,
                           ctypes.c_int64, vp, vp]
        lib.oracle_op_size.restype = ctypes.c_int64
        lib.oracle_op_size.argtypes = [vp]
        lib.oracle_op_export.restype = None
        lib.oracle_op_export.argtypes = [vp, vp, vp]
        lib.oracle_op_free.restype = None
        lib.oracle_op_free.argtypes = [vp]
        _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# operators as {label: complex}
# ---------------------------------------------------------------------------
def _arrays(op):
    labels = np.fromiter((int(k) for k in op.keys()), dtype=np.uint64, count=len(op))
    coefs = np.empty(2 * len(op))
    vals = np.fromiter((complex(v) for v in op.values()), dtype=np.complex128, count=len(op))
    coefs[0::2] = vals.real
    coefs[1::2] = vals.imag
    return labels, coefs


def _call(fn_name, alg, nmodes, A, B):
    lib = _load()
    la, ca = _arrays(A)
    lb, cb = _arrays(B)
    h = getattr(lib, fn_name)(alg, nmodes, len(la), la.ctypes.data, ca.ctypes.data,
                              len(lb), lb.ctypes.data, cb.ctypes.data)
    try:
        n = lib.oracle_op_size(h)
        labels = np.empty(n, dtype=np.uint64)
        coefs = np.empty(2 * n)
        lib.oracle_op_export(h, labels.ctypes.data, coefs.ctypes.data)
    finally:
        lib.oracle_op_free(h)
    return {int(l): complex(coefs[2 * i], coefs[2 * i + 1]) for i, l in enumerate(labels)}


def product(alg, nmodes, A, B):
    """Exact product A*B (Sec. 2.1: evaluated in the full algebra, normal ordered)."""
    return _call("oracle_product", alg, nmodes, A, B)


def commutator(alg, nmodes, A, B):
    """Exact, unprojected commutator [A, B]."""
    return _call("oracle_commutator", alg, nmodes, A, B)


def is_diagonal(alg, label):
    """The diagonal mask D of Sec. 2.2."""
    label = int(label)
    lo, hi = label & 0xFFFFFFFF, label >> 32
    if alg == ALG_PAULI:
        return lo == 0                 # no X or Y factor
    if alg == ALG_PAULI_BOSON:         # I or Z Pauli factor, c = a in every mode
        if (label & 3) in (1, 2):
            return False
        return all(((label >> (2 + 10 * m)) & 31) == ((label >> (7 + 10 * m)) & 31) for m in range(6))
    return lo == hi                    # creator set == annihilator set


def as_operator(labels, coefs):
    return {int(l): complex(c) for l, c in zip(labels, coefs) if c != 0}


def project(op, labels):
    """P: keep the registry coordinates (complex)."""
    return np.array([op.get(int(l), 0.0) for l in labels], dtype=np.complex128)


def _real(v, what):
    v = np.asarray(v, dtype=np.complex128)
    scale = max(1.0, float(np.max(np.abs(v))) if v.size else 1.0)
    if v.size and np.max(np.abs(v.imag)) > 1e-9 * scale:
        raise AssertionError(f"{what}: imaginary part {np.max(np.abs(v.imag))} in a real coordinate")
    return v.real.copy()


def generator(alg, nmodes, labels, h):
    """eta = [H_d, H_od] as {label: complex} (Eq. block-generator)."""
    Hd = {int(l): complex(c) for l, c in zip(labels, h) if c != 0 and is_diagonal(alg, l)}
    Hod = {int(l): complex(c) for l, c in zip(labels, h) if c != 0 and not is_diagonal(alg, l)}
    return commutator(alg, nmodes, Hd, Hod)


def xi_of(alg, eta):
    """Real generator coordinates: eta = i sum xi G (Pauli), sum xi G (fermion)."""
    if alg == ALG_PAULI:
        return {k: (v / 1j) for k, v in eta.items()}
    return dict(eta)


def rhs(alg, nmodes, labels, h, xs=(), return_eta=False):
    """dh = P[eta(h), H], dx_o = P[eta(h), X_o]  (Eqs. coflow, projected-flow)."""
    eta = generator(alg, nmodes, labels, h)
    out = []
    for v in [h] + list(xs):
        F = commutator(alg, nmodes, eta, as_operator(labels, v))
        out.append(_real(project(F, labels), "rhs"))
    if return_eta:
        return out[0], out[1:], eta
    return out[0], out[1:]


def rhs_unprojected(alg, nmodes, labels, h, x):
    """[eta(h), X] before the projection P (for the dense-matrix pins)."""
    eta = generator(alg, nmodes, labels, h)
    return commutator(alg, nmodes, eta, as_operator(labels, x))


def rhs_vjp(alg, nmodes, labels, h, xs, w_h, w_xs):
    """Vector-Jacobian product of the right-hand side (Sec. 2.4, adjoint traversal).

    With F_o = P[eta(h), X_o] (X_0 = H) and the scalar
    L = sum_o <w_o, F_o>, returns (h_bar, [x_bar_o]) = (dL/dh, dL/dx_o), by
    the chain rule through the string algebra:
      x_bar_o[j] = <w_o, P[eta, O_j]>
      c_g        = sum_o <w_o, P[G_g, X_o]>          (dL/d eta_g)
      h_bar[i]   = Re sum_g c_g d(eta_g)/d(h_i) + x_bar_0[i],
    where d eta/d h_i = [O_i, H_od] for diagonal i and [H_d, O_i] otherwise.
    """
    labels = [int(l) for l in labels]
    n = len(labels)
    operands = [np.asarray(h)] + [np.asarray(x) for x in xs]
    weights = [np.asarray(w_h)] + [np.asarray(w) for w in w_xs]
    diag = [is_diagonal(alg, l) for l in labels]
    Hd = {l: complex(c) for l, c, d in zip(labels, h, diag) if c != 0 and d}
    Hod = {l: complex(c) for l, c, d in zip(labels, h, diag) if c != 0 and not d}
    eta = commutator(alg, nmodes, Hd, Hod)

    # operand adjoints: x_bar_o[j] = <w_o, P[eta, O_j]>
    cols = np.zeros((n, n), dtype=np.complex128)      # cols[j] = P[eta, O_j]
    for j, l in enumerate(labels):
        cols[j] = project(commutator(alg, nmodes, eta, {l: 1.0}), labels)
    x_bar = [cols @ w for w in weights]

    X_ops = [as_operator(labels, v) for v in operands]
    cache = {}

    def c_of(g):
        if g not in cache:
            s = 0.0
            for Xo, wo in zip(X_ops, weights):
                s += project(commutator(alg, nmodes, {g: 1.0}, Xo), labels) @ wo
            cache[g] = s
        return cache[g]

    h_bar = np.zeros(n, dtype=np.complex128)
    for i, l in enumerate(labels):
        if diag[i]:
            d_eta = commutator(alg, nmodes, {l: 1.0}, Hod)
        else:
            d_eta = commutator(alg, nmodes, Hd, {l: 1.0})
        h_bar[i] = sum(c_of(g) * v for g, v in d_eta.items() if v != 0)
    h_bar += x_bar[0]
    return _real(h_bar, "h_bar"), [_real(v, "x_bar") for v in x_bar[1:]]


def rhs_jvp(alg, nmodes, labels, h, xs, dh, dxs, eps=0.25):
    """Directional derivative of the right-hand side (Sec. 2.4, Eq.
    directional-derivative).  The right-hand side is a polynomial of degree 3
    in (h, x), so the five-point central formula
    (-f(2e) + 8 f(e) - 8 f(-e) + f(-2e)) / (12 e) is exact up to rounding."""
    h = np.asarray(h, dtype=np.float64)
    dh = np.asarray(dh, dtype=np.float64)
    xs = [np.asarray(x, dtype=np.float64) for x in xs]
    dxs = [np.asarray(x, dtype=np.float64) for x in dxs]

    def f(t):
        a, b = rhs(alg, nmodes, labels, h + t * dh, [x + t * d for x, d in zip(xs, dxs)])
        return [a] + list(b)
    fm2, fm1, fp1, fp2 = f(-2 * eps), f(-eps), f(eps), f(2 * eps)
    out = [(-p2 + 8 * p1 - 8 * m1 + m2) / (12 * eps) for m2, m1, p1, p2 in zip(fm2, fm1, fp1, fp2)]
    return out[0], out[1:]


# ---------------------------------------------------------------------------
# flows on the stacked state y = [h; x_1; ...; x_m]
# ---------------------------------------------------------------------------
def stacked_rhs(alg, nmodes, labels, n_obs):
    n = len(labels)

    def f(y):
        h = y[:n]
        xs = [y[(o + 1) * n:(o + 2) * n] for o in range(n_obs)]
        dh, dxs = rhs(alg, nmodes, labels, h, xs)
        return np.concatenate([dh] + dxs)
    return f


def stacked_vjp(alg, nmodes, labels, n_obs):
    n = len(labels)

    def fv(y, w):
        h = y[:n]
        xs = [y[(o + 1) * n:(o + 2) * n] for o in range(n_obs)]
        wh = w[:n]
        wx = [w[(o + 1) * n:(o + 2) * n] for o in range(n_obs)]
        hb, xb = rhs_vjp(alg, nmodes, labels, h, xs, wh, wx)
        return np.concatenate([hb] + xb)
    return fv


# classical fourth-order Runge-Kutta tableau
RK4_A = [[], [0.5], [0.0, 0.5], [0.0, 0.0, 1.0]]
RK4_B = [1 / 6, 1 / 3, 1 / 3, 1 / 6]

# Dormand-Prince 5(4) tableau (Dormand & Prince, J. Comput. Appl. Math. 6, 1980)
DP_A = [[],
        [1 / 5],
        [3 / 40, 9 / 40],
        [44 / 45, -56 / 15, 32 / 9],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
        [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]]
DP_B = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0]
DP_BSTAR = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]


def rk_step(f, y, ds, A, B):
    """One explicit Runge-Kutta step; returns (y_new, stage inputs, stage slopes)."""
    ks, us = [], []
    for i in range(len(B)):
        u = y.copy()
        for j, a in enumerate(A[i]):
            if a != 0.0:
                u = u + ds * a * ks[j]
        us.append(u)
        ks.append(f(u))
    y_new = y.copy()
    for b, k in zip(B, ks):
        if b != 0.0:
            y_new = y_new + ds * b * k
    return y_new, us, ks


def rk4_flow(f, y0, ds, nsteps):
    y = np.array(y0, dtype=np.float64)
    for _ in range(nsteps):
        y, _, _ = rk_step(f, y, ds, RK4_A, RK4_B)
    return y


def dp45_flow(f, y0, s0, s1, ds0, rtol, atol, max_steps=100000, replay=None):
    """Adaptive Dormand-Prince 5(4).

    Controller (a reading; the workloads fix only rtol): error ratio
    r = max_k |e_k| / (atol + rtol max(|y_k|, |y5_k|)); accept when r <= 1;
    ds <- ds * clamp(0.9 r^(-1/5), 0.2, 5) (growth capped at 1 after a
    rejection); the last step is shortened to land on s1.
    With `replay` (a list of accepted step sizes) every listed step is taken
    and accepted as given, so that two implementations follow one path.
    Returns (y, accepted_steps, n_rejected).
    """
    y = np.array(y0, dtype=np.float64)
    A = DP_A[:6]
    B6 = DP_B[:6]
    if replay is not None:
        for ds in replay:
            y, _, _ = rk_step(f, y, ds, A, B6)
        return y, list(replay), 0
    s, ds = s0, ds0
    accepted, rejected = [], 0
    while s < s1 and len(accepted) + rejected < max_steps:
        ds = min(ds, s1 - s)
        y5, _, ks = rk_step(f, y, ds, A, B6)
        k7 = f(y5)
        ks = ks + [k7]
        err = np.zeros_like(y)
        for b, bs, k in zip(DP_B, DP_BSTAR, ks):
            if b - bs != 0.0:
                err = err + ds * (b - bs) * k
        scale = atol + rtol * np.maximum(np.abs(y), np.abs(y5))
        r = float(np.max(np.abs(err) / scale))
        if r <= 1.0:
            s += ds
            y = y5
            accepted.append(ds)
            fac = 5.0 if r == 0.0 else min(5.0, max(0.2, 0.9 * r ** -0.2))
        else:
            rejected += 1
            fac = min(1.0, max(0.2, 0.9 * r ** -0.2))
        ds = ds * fac
    return y, accepted, rejected


def rk_flow_vjp(f, fv, y0, steps, A, B, y_bar_final):
    """Discrete adjoint of an explicit RK trajectory with the given step sizes.

    Stage by stage, in reverse: k_bar_i starts at ds b_i y_bar; for each
    stage i (last first) u_bar_i = J(u_i)^T k_bar_i is added to y_bar and
    ds a_ij u_bar_i to k_bar_j (j < i).  Returns (y_final, y_bar(0)).
    """
    ys, stages = [np.array(y0, dtype=np.float64)], []
    for ds in steps:
        y_new, us, _ = rk_step(f, ys[-1], ds, A, B)
        stages.append(us)
        ys.append(y_new)
    yb = np.array(y_bar_final, dtype=np.float64)
    for ds, us in zip(reversed(steps), reversed(stages)):
        kb = [ds * b * yb for b in B]
        yb_new = yb.copy()
        for i in reversed(range(len(B))):
            if not np.any(kb[i]):
                continue
            ub = fv(us[i], kb[i])
            yb_new = yb_new + ub
            for j, a in enumerate(A[i]):
                if a != 0.0:
                    kb[j] = kb[j] + ds * a * ub
        yb = yb_new
    return ys[-1], yb

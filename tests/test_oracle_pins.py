"""Pins of the CPU oracle against things other than itself (CPU only).

Each check fixes a part of the oracle that a plausible mistake would break:
textbook identities (golden fixture), dense Kronecker / Jordan-Wigner matrix
products, dense Wegner flows that the projected coefficient flow must
reproduce exactly (closed Pauli algebra; fermion particle-number sectors),
invariants of the flow, exact polynomial derivatives for the adjoint, and
order conditions / closed-form ODEs for the integrators.
"""
import json
import os
from itertools import combinations

import numpy as np
import pytest

import oracle
from cut_inputs import (ALG_FERMION, ALG_PAULI, fermion_registry, make_label,
                        molecular_hamiltonian, number_operator, dipole_operator,
                        pauli_registry, workload)
from cut_inputs.registry import pauli_label
import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "algebra_identities.jsonl")


def _fermion_label(text):
    cre, ann = [], []
    for tok in text.split():
        if tok.startswith("a+"):
            cre.append(int(tok[2:]))
        else:
            ann.append(int(tok[1:]))
    assert cre == sorted(cre) and ann == sorted(ann, reverse=True), text
    return make_label(sum(1 << p for p in cre), sum(1 << p for p in ann))


def _label(alg, text):
    if alg == "pauli":
        return pauli_label(text)
    if text == "":
        return 0
    return _fermion_label(text)


def test_golden_identities():
    with open(GOLDEN) as f:
        cases = [json.loads(l) for l in f if l.strip()]
    assert len(cases) >= 15
    for c in cases:
        alg = ALG_PAULI if c["alg"] == "pauli" else ALG_FERMION
        a = {_label(c["alg"], c["a"]): 1.0}
        b = {_label(c["alg"], c["b"]): 1.0}
        fn = oracle.product if c["op"] == "prod" else oracle.commutator
        got = {k: v for k, v in fn(alg, c["nmodes"], a, b).items() if v != 0}
        want = {_label(c["alg"], t): complex(re, im) for t, re, im in c["result"]}
        assert got == want, (c, got)


def _dense_check(alg, nmodes, labels, pairs, fn, dfn):
    for la, lb in pairs:
        got = fn(alg, nmodes, {int(la): 1.0}, {int(lb): 1.0})
        M = dense.op_matrix(got, alg, nmodes)
        f = dense.pauli_matrix if alg == ALG_PAULI else dense.fermion_matrix
        A, B = f(la, nmodes), f(lb, nmodes)
        np.testing.assert_allclose(M, dfn(A, B), atol=1e-13)


def test_pauli_products_match_kronecker_matrices():
    labels = pauli_registry(2)
    pairs = [(a, b) for a in labels for b in labels]
    _dense_check(ALG_PAULI, 2, labels, pairs, oracle.product, lambda A, B: A @ B)
    rng = np.random.default_rng(5)
    labels3 = pauli_registry(3)
    pairs = [tuple(rng.choice(labels3, 2)) for _ in range(60)]
    _dense_check(ALG_PAULI, 3, labels3, pairs, oracle.commutator, lambda A, B: A @ B - B @ A)


def test_fermion_products_match_jordan_wigner():
    labels = fermion_registry(3, ranks=(1, 2, 3))
    pairs = [(a, b) for a in labels for b in labels]
    _dense_check(ALG_FERMION, 3, labels, pairs, oracle.product, lambda A, B: A @ B)
    rng = np.random.default_rng(6)
    labels5 = fermion_registry(5, ranks=(1, 2, 3))
    pairs = [tuple(rng.choice(labels5, 2)) for _ in range(80)]
    _dense_check(ALG_FERMION, 5, labels5, pairs, oracle.commutator, lambda A, B: A @ B - B @ A)


def test_pauli_rhs_matches_dense_commutators():
    """Closed algebra: P is the identity, so dH = [[H_d, H_od], H] exactly."""
    nq = 3
    labels = pauli_registry(nq)
    rng = np.random.default_rng(7)
    h = rng.normal(size=len(labels))          # any real vector is a Hermitian H
    x = rng.normal(size=len(labels))
    dh, (dx,) = oracle.rhs(ALG_PAULI, nq, labels, h, [x])
    H = dense.vec_matrix(labels, h, ALG_PAULI, nq)
    X = dense.vec_matrix(labels, x, ALG_PAULI, nq)
    Hd = np.diag(np.diag(H))                  # I/Z strings are the diagonal
    eta = Hd @ H - H @ Hd
    np.testing.assert_allclose(dh, dense.pauli_coefficients(eta @ H - H @ eta, labels, nq).real, atol=1e-12)
    np.testing.assert_allclose(dx, dense.pauli_coefficients(eta @ X - X @ eta, labels, nq).real, atol=1e-12)
    # generator coordinates: eta = i sum xi G
    _, _, eta_op = oracle.rhs(ALG_PAULI, nq, labels, h, [], return_eta=True)
    xi = oracle.xi_of(ALG_PAULI, eta_op)
    want = dense.pauli_coefficients(eta, labels, nq) / 1j
    got = np.array([xi.get(int(l), 0.0) for l in labels])
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_fermion_unprojected_commutator_matches_jordan_wigner():
    norb = 5
    labels = fermion_registry(norb, ranks=(1, 2))
    rng = np.random.default_rng(8)
    h = molecular_hamiltonian(labels, norb, seed=8, scale=0.3)
    x = dipole_operator(labels, norb, seed=8)
    F = oracle.rhs_unprojected(ALG_FERMION, norb, labels, h, x)
    H = dense.vec_matrix(labels, h, ALG_FERMION, norb)
    X = dense.vec_matrix(labels, x, ALG_FERMION, norb)
    # D selects n_p and n_p n_q: exactly the diagonal of H in the occupation basis
    Hd = np.diag(np.diag(H))
    eta = Hd @ H - H @ Hd
    np.testing.assert_allclose(dense.op_matrix(F, ALG_FERMION, norb), eta @ X - X @ eta, atol=1e-12)


def _sector_blocks(labels, v, norb):
    M = dense.vec_matrix(labels, v, ALG_FERMION, norb)
    return [dense.sector_block(M, norb, N) for N in (1, 2)]


def test_fermion_projected_rhs_equals_sector_wegner_rhs():
    """Rank >= 3 terms annihilate every state with <= 2 particles, so the
    projected <=2-body right-hand side restricted to the N=1 and N=2 sectors
    is the dense Wegner right-hand side of those blocks."""
    norb = 5
    labels = fermion_registry(norb, ranks=(1, 2))
    h = molecular_hamiltonian(labels, norb, seed=9, scale=0.2)
    x = dipole_operator(labels, norb, seed=9)
    dh, (dx,) = oracle.rhs(ALG_FERMION, norb, labels, h, [x])
    for B, X, dB, dX in zip(_sector_blocks(labels, h, norb), _sector_blocks(labels, x, norb),
                            _sector_blocks(labels, dh, norb), _sector_blocks(labels, dx, norb)):
        want, eta = dense.wegner_rhs(B)
        np.testing.assert_allclose(dB, want, atol=1e-12)
        np.testing.assert_allclose(dX, eta @ X - X @ eta, atol=1e-12)


def test_generator_truncation_lemma():
    """Generator terms of rank > 2 never reach the rank <= 2 registry."""
    norb = 5
    labels = fermion_registry(norb, ranks=(1, 2))
    h = molecular_hamiltonian(labels, norb, seed=10, scale=0.3)
    eta = oracle.generator(ALG_FERMION, norb, labels, h)
    ranks = {bin(k & 0xFFFFFFFF).count("1") for k, v in eta.items() if v != 0}
    assert 3 in ranks                       # the lemma is not vacuous here
    low = {k: v for k, v in eta.items() if bin(k & 0xFFFFFFFF).count("1") <= 2}
    Hop = oracle.as_operator(labels, h)
    full = oracle.project(oracle.commutator(ALG_FERMION, norb, eta, Hop), labels)
    trunc = oracle.project(oracle.commutator(ALG_FERMION, norb, low, Hop), labels)
    np.testing.assert_allclose(full, trunc, rtol=0, atol=1e-14)


def test_diagonal_hamiltonian_has_zero_generator_and_rhs():
    labels, h = pauli_registry(3), None
    rng = np.random.default_rng(11)
    h = np.array([rng.normal() if oracle.is_diagonal(ALG_PAULI, l) else 0.0 for l in labels])
    dh, _ = oracle.rhs(ALG_PAULI, 3, labels, h)
    assert np.all(dh == 0.0)
    labels = fermion_registry(4)
    h = np.array([rng.normal() if oracle.is_diagonal(ALG_FERMION, l) else 0.0 for l in labels])
    eta = oracle.generator(ALG_FERMION, 4, labels, h)
    assert all(v == 0 for v in eta.values())
    dh, _ = oracle.rhs(ALG_FERMION, 4, labels, h)
    assert np.all(dh == 0.0)


def test_pauli_flow_matches_dense_wegner_flow_and_invariants():
    """Closed 4-qubit algebra: the coefficient flow is the 16x16 Wegner flow."""
    w = workload("closed_pauli_4q")
    f = oracle.stacked_rhs(w.alg, w.nmodes, w.labels, 0)
    nsteps = 60
    y = oracle.rk4_flow(f, w.h, w.ds, nsteps)
    H0 = dense.vec_matrix(w.labels, w.h, ALG_PAULI, 4)
    Hs = dense.rk4_dense(lambda B: dense.wegner_rhs(B)[0], H0, w.ds, nsteps)
    np.testing.assert_allclose(dense.pauli_coefficients(Hs, w.labels, 4).real, y, atol=1e-11)
    # spectrum, Tr H^2 = 16 sum c^2, Wegner decay of the off-diagonal norm, odd-Y zero
    # RK4 keeps the spectrum and Tr H^2 only to its truncation error at this ds
    Hy = dense.vec_matrix(w.labels, y, ALG_PAULI, 4)
    np.testing.assert_allclose(np.linalg.eigvalsh(Hy), np.linalg.eigvalsh(H0), rtol=1e-5)
    np.testing.assert_allclose(np.sum(y ** 2), np.sum(w.h ** 2), rtol=1e-6)
    # ... while the right-hand side itself is exactly isospectral: Tr(H^k dH) = 0
    dh = f(w.h)
    dH = dense.vec_matrix(w.labels, dh, ALG_PAULI, 4)
    for k in (0, 1, 2, 3):
        Hk = np.linalg.matrix_power(H0, k)
        assert abs(np.trace(Hk @ dH)) < 1e-12 * np.linalg.norm(Hk) * np.linalg.norm(dH) * 16
    od = np.array([not oracle.is_diagonal(ALG_PAULI, l) for l in w.labels])
    odd_y = np.array([bin((int(l) & 0xFFFFFFFF) & (int(l) >> 32)).count("1") % 2 == 1 for l in w.labels])
    assert np.sum(y[od] ** 2) < np.sum(w.h[od] ** 2)
    assert np.all(y[odd_y] == 0.0)


def test_fermion_flow_matches_sector_wegner_flows():
    """Projected <=2-body flow == dense Wegner flows of the N=1, N=2 blocks;
    the particle number N is carried unchanged."""
    norb = 4
    labels = fermion_registry(norb)
    h = molecular_hamiltonian(labels, norb, seed=12, scale=0.2)
    N = number_operator(labels, norb)
    D = dipole_operator(labels, norb, seed=12)
    n = len(labels)
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 2)
    ds, nsteps = 0.02, 25
    y = oracle.rk4_flow(f, np.concatenate([h, N, D]), ds, nsteps)
    np.testing.assert_array_equal(y[n:2 * n], N)
    blocks0 = _sector_blocks(labels, h, norb)
    blocksD = _sector_blocks(labels, D, norb)
    got_h = _sector_blocks(labels, y[:n], norb)
    got_D = _sector_blocks(labels, y[2 * n:], norb)

    def pair_rhs(BX):
        B, X = BX
        dB, eta = dense.wegner_rhs(B)
        return np.stack([dB, eta @ X - X @ eta])

    for B0, X0, Bs, Xs in zip(blocks0, blocksD, got_h, got_D):
        out = dense.rk4_dense(pair_rhs, np.stack([B0, X0]), ds, nsteps)
        np.testing.assert_allclose(Bs, out[0], atol=1e-12)
        np.testing.assert_allclose(Xs, out[1], atol=1e-12)
        # the spectrum is kept to the RK4 truncation error at this step size
        np.testing.assert_allclose(np.linalg.eigvalsh(Bs), np.linalg.eigvalsh(B0), rtol=1e-5)


def _five_point(f, y, v, eps=0.25):
    """Derivative of a polynomial of degree <= 4 along v: exact up to rounding."""
    return (-f(y + 2 * eps * v) + 8 * f(y + eps * v) - 8 * f(y - eps * v) + f(y - 2 * eps * v)) / (12 * eps)


@pytest.mark.parametrize("alg,nmodes", [(ALG_PAULI, 2), (ALG_FERMION, 3)])
def test_rhs_vjp_pairs_with_exact_directional_derivative(alg, nmodes):
    labels = pauli_registry(nmodes) if alg == ALG_PAULI else fermion_registry(nmodes)
    n = len(labels)
    rng = np.random.default_rng(13)
    y = rng.normal(size=3 * n)
    v = rng.normal(size=3 * n)
    w = rng.normal(size=3 * n)
    f = oracle.stacked_rhs(alg, nmodes, labels, 2)
    fv = oracle.stacked_vjp(alg, nmodes, labels, 2)
    jv = _five_point(f, y, v)
    jtw = fv(y, w)
    np.testing.assert_allclose(w @ jv, jtw @ v, rtol=1e-12)
    # full Jacobian transpose, column by column on the h block
    for k in range(0, n, max(1, n // 5)):
        e = np.zeros(3 * n)
        e[k] = 1.0
        np.testing.assert_allclose(w @ _five_point(f, y, e), jtw[k], rtol=1e-10, atol=1e-12)


def test_flow_vjp_matches_central_differences():
    norb = 3
    labels = fermion_registry(norb)
    n = len(labels)
    h = molecular_hamiltonian(labels, norb, seed=14, scale=0.3)
    D = dipole_operator(labels, norb, seed=14)
    y0 = np.concatenate([h, D])
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 1)
    fv = oracle.stacked_vjp(ALG_FERMION, norb, labels, 1)
    steps = [0.05] * 6
    target = n  # first coefficient of the carried observable
    yb = np.zeros(2 * n)
    yb[target] = 1.0
    _, grad = oracle.rk_flow_vjp(f, fv, y0, steps, oracle.RK4_A, oracle.RK4_B, yb)
    rng = np.random.default_rng(15)
    for _ in range(3):
        v = rng.normal(size=2 * n)
        eps = 1e-5
        yp = oracle.rk4_flow(f, y0 + eps * v, 0.05, 6)
        ym = oracle.rk4_flow(f, y0 - eps * v, 0.05, 6)
        fd = (yp[target] - ym[target]) / (2 * eps)
        np.testing.assert_allclose(grad @ v, fd, rtol=1e-7, atol=1e-10)


def test_integrator_tableaux_and_closed_form_odes():
    for A, B in ((oracle.RK4_A, oracle.RK4_B), (oracle.DP_A[:6], oracle.DP_B[:6])):
        c = [sum(r) for r in A]
        assert abs(sum(B) - 1) < 1e-15
        assert abs(sum(b * ci for b, ci in zip(B, c)) - 0.5) < 1e-15
        assert abs(sum(b * ci ** 2 for b, ci in zip(B, c)) - 1 / 3) < 1e-15
        assert abs(sum(b * ci ** 3 for b, ci in zip(B, c)) - 1 / 4) < 1e-15
    assert abs(sum(oracle.DP_BSTAR) - 1) < 1e-15
    # RK4 on y' = -y: error 1e-12-ish at ds 1e-2
    y = oracle.rk4_flow(lambda y: -y, np.array([1.0]), 0.01, 100)
    assert abs(y[0] - np.exp(-1.0)) < 1e-9
    # DP45 on y' = A y with a rotation + decay, against expm
    A = np.array([[-0.5, 2.0], [-2.0, -0.5]])
    y, steps, rej = oracle.dp45_flow(lambda y: A @ y, np.array([1.0, 0.0]), 0.0, 3.0, 0.1, 1e-10, 1e-14)
    from scipy.linalg import expm
    np.testing.assert_allclose(y, expm(3.0 * A) @ np.array([1.0, 0.0]), rtol=1e-8, atol=1e-10)
    assert abs(sum(steps) - 3.0) < 1e-12 and len(steps) > 10
    # replay of the accepted steps reproduces the result exactly
    y2, _, _ = oracle.dp45_flow(lambda y: A @ y, np.array([1.0, 0.0]), 0.0, 3.0, 0.1, 1e-10, 1e-14, replay=steps)
    np.testing.assert_array_equal(y, y2)


def test_occupation_sector_matrices_match_jordan_wigner_blocks():
    """The occupation-basis sector helper used by the full-size GPU flow
    checks agrees with the Jordan-Wigner matrices."""
    norb = 5
    labels = fermion_registry(norb, ranks=(1, 2, 3))
    h = molecular_hamiltonian(labels, norb, seed=16, scale=0.3)
    M = dense.vec_matrix(labels, h, ALG_FERMION, norb)
    for N in (1, 2, 3):
        np.testing.assert_allclose(dense.sector_matrix(labels, h, norb, N), dense.sector_block(M, norb, N).real,
                                   atol=1e-13)


def test_mlp_oracle_gradients_match_central_differences():
    """Pins the oracle MLP's chain rule (FP64, no rounding emulation)."""
    from oracle import mlp
    rng = np.random.default_rng(40)
    n_in, n_hid, n_out, B = 5, 7, 4, 6
    layers = [(rng.normal(size=(n_hid, n_in)) * 0.5, rng.normal(size=n_hid) * 0.1),
              (rng.normal(size=(n_hid, n_hid)) * 0.4, rng.normal(size=n_hid) * 0.1),
              (rng.normal(size=(n_out, n_hid)) * 0.4, rng.normal(size=n_out) * 0.1)]
    X = rng.normal(size=(B, n_in))
    T = rng.normal(size=(B, n_out))
    scale, shift = rng.uniform(0.5, 2.0, n_out), rng.normal(size=n_out)
    loss, grads = mlp.loss_and_grads(layers, X, T, scale, shift, emulate=False)
    flat = mlp.flatten(layers)
    g = mlp.flatten(grads)
    for k in rng.choice(flat.size, 25, replace=False):
        e = np.zeros_like(flat)
        e[k] = 1e-6
        lp, _ = mlp.loss_and_grads(mlp.unflatten(flat + e, n_in, n_hid, n_out), X, T, scale, shift, emulate=False)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(flat - e, n_in, n_hid, n_out), X, T, scale, shift, emulate=False)
        np.testing.assert_allclose(g[k], (lp - lm) / 2e-6, rtol=1e-6, atol=1e-10)
    # GELU against its closed-form values and bf16 rounding against exact cases
    np.testing.assert_allclose(mlp.gelu(np.array([0.0, 1.0, -1.0])), [0.0, 0.8413447460685429, -0.15865525393145707],
                               rtol=1e-15)
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0                 # tie -> even
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert mlp.bf16(np.array([1.0 + 2.0 ** -7]))[0] == 1.0 + 2.0 ** -7      # representable


def test_oracle_jvp_pairs_with_vjp():
    """<w, J v> from the exact five-point tangent equals <J^T w, v>."""
    labels = fermion_registry(3)
    n = len(labels)
    rng = np.random.default_rng(17)
    h, x = rng.normal(size=n), rng.normal(size=n)
    dh, dx = rng.normal(size=n), rng.normal(size=n)
    wh, wx = rng.normal(size=n), rng.normal(size=n)
    jh, (jx,) = oracle.rhs_jvp(ALG_FERMION, 3, labels, h, [x], dh, [dx])
    bh, (bx,) = oracle.rhs_vjp(ALG_FERMION, 3, labels, h, [x], wh, [wx])
    np.testing.assert_allclose(wh @ jh + wx @ jx, bh @ dh + bx @ dx, rtol=1e-12)


def test_adamw_oracle_worked_example_and_special_cases():
    """Pins the oracle's AdamW step (Loshchilov & Hutter, decoupled weight
    decay) against a hand-worked two-step example and against special cases
    that a plausible mistake breaks.

    Worked example, p0 = 1, lr = 0.1, beta1 = 0.9, beta2 = 0.999,
    eps = 1e-8, wd = 0.01, m0 = v0 = 0:
      t = 1, g = 0.5:  m = 0.1 * 0.5 = 0.05;  v = 0.001 * 0.25 = 2.5e-4;
        m_hat = 0.05 / (1 - 0.9) = 0.5;  v_hat = 2.5e-4 / (1 - 0.999) = 0.25;
        p1 = 1 - 0.1 * (0.5 / (0.5 + 1e-8) + 0.01 * 1) = 0.899000002 (to 1e-16)
      t = 2, g = -0.25:  m = 0.9 * 0.05 + 0.1 * (-0.25) = 0.02;
        v = 0.999 * 2.5e-4 + 0.001 * 0.0625 = 3.1225e-4;
        m_hat = 0.02 / (1 - 0.81) = 2/19;  v_hat = 3.1225e-4 / (1 - 0.998001);
        p2 = p1 - 0.1 * (m_hat / (sqrt(v_hat) + 1e-8) + 0.01 * p1)
           = 0.871467298705846163 (40-digit decimal arithmetic)
    """
    from oracle import mlp
    p, m, v = mlp.adamw(np.array([1.0]), np.array([0.5]), 0.0, 0.0, 1, 0.1, 0.9, 0.999, 1e-8, 0.01)
    np.testing.assert_allclose(m, [0.05], rtol=1e-15)
    np.testing.assert_allclose(v, [2.5e-4], rtol=1e-14)
    np.testing.assert_allclose(p, [0.8990000019999999600], rtol=1e-15)
    p, m, v = mlp.adamw(p, np.array([-0.25]), m, v, 2, 0.1, 0.9, 0.999, 1e-8, 0.01)
    np.testing.assert_allclose(m, [0.02], rtol=1e-14)
    np.testing.assert_allclose(v, [3.1225e-4], rtol=1e-14)
    np.testing.assert_allclose(p, [0.8714672987058461626], rtol=1e-15)

    g = np.array([3.0, -1e-3, 40.0])
    # bias correction: the first step from zero moments moves every
    # parameter by lr * sign(g) (up to eps), whatever |g| is
    p1, _, _ = mlp.adamw(np.zeros(3), g, 0.0, 0.0, 1, 0.01, 0.9, 0.999, 1e-12, 0.0)
    np.testing.assert_allclose(p1, -0.01 * np.sign(g), rtol=1e-8)
    # decoupled decay, scaled by lr: with no gradient p -> p (1 - lr wd),
    # and the moments stay zero (an L2 penalty would have entered them)
    p1, m1, v1 = mlp.adamw(np.array([2.0]), np.array([0.0]), 0.0, 0.0, 1, 0.1, 0.9, 0.999, 1e-8, 0.5)
    np.testing.assert_allclose(p1, [2.0 * (1 - 0.1 * 0.5)], rtol=1e-15)
    assert m1[0] == 0.0 and v1[0] == 0.0
    # eps outside the square root: g = eps gives m_hat / (|g| + eps) = 1/2
    p1, _, _ = mlp.adamw(np.array([0.0]), np.array([1e-8]), 0.0, 0.0, 1, 1.0, 0.9, 0.999, 1e-8, 0.0)
    np.testing.assert_allclose(p1, [-0.5], rtol=1e-12)

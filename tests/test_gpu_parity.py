"""CUDA path against the oracle, element by element (needs a B300).

Tolerance: RTOL = 1e-10 relative (FP64), see gpu_util.assert_close.  Full
sizes where the oracle is fast enough (closed 4-qubit Pauli algebra,
8-spin-orbital molecular model: one right-hand side each); flows at full
size are checked through properties that hold at any size (the exact
equivalence with dense Wegner flows of the closed algebra / the N=1 and N=2
sectors) and against the oracle on smaller registries.
"""
import numpy as np
import pytest

import oracle
import dense
from gpu_util import assert_close, graph_for, np64, rhs_floor
from cut_inputs import (ALG_FERMION, ALG_PAULI, cfg2_registry, dipole_operator, fermion_registry,
                        molecular_hamiltonian, number_operator, pauli_registry, workload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_14831_b300 import build
    build.build()


def _case(name):
    if name == "pauli4":
        w = workload("closed_pauli_4q")
        rng = np.random.default_rng(21)
        return w.alg, w.nmodes, w.labels, w.h, [rng.normal(size=len(w.labels))]
    if name == "mol8":
        w = workload("molecular_8so")
        return w.alg, w.nmodes, w.labels, w.h, w.observables
    if name == "mol5_3body":
        labels = cfg2_registry(5, keep_shared1=0.3, seed=3)
        h = molecular_hamiltonian(labels, 5, seed=22, scale=0.3)
        return ALG_FERMION, 5, labels, h, [number_operator(labels, 5), dipole_operator(labels, 5, seed=22)]
    if name == "pauli3_ragged":
        labels = pauli_registry(3)[::3]          # a non-closed registry with a ragged tail
        rng = np.random.default_rng(23)
        return ALG_PAULI, 3, labels, rng.normal(size=len(labels)), []
    raise KeyError(name)


def _xi_oracle(alg, eta, gen_labels):
    xi = oracle.xi_of(alg, eta)
    return np.array([complex(xi.get(int(g), 0.0)).real for g in gen_labels])


@pytest.mark.parametrize("name", ["pauli4", "mol8", "mol5_3body", "pauli3_ragged"])
def test_rhs_matches_oracle(name):
    alg, nm, labels, h, xs = _case(name)
    G = graph_for(name, alg, nm, labels)
    dh, dxs, xi = G.rhs(h, xs, want_xi=True)
    want_dh, want_dxs, eta = oracle.rhs(alg, nm, labels, h, xs, return_eta=True)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what="dh", atol=fl)
    for got, want in zip(dxs, want_dxs):
        assert_close(np64(got), want, what="dx", atol=fl)
    _, gen_labels, _ = G.labels()
    assert_close(np64(xi), _xi_oracle(alg, eta, gen_labels), what="xi")


def test_rhs_is_bitwise_deterministic_and_n_obs_independent():
    alg, nm, labels, h, xs = _case("mol8")
    G = graph_for("mol8", alg, nm, labels)
    a = G.rhs(h, xs)
    b = G.rhs(h, xs)
    c = G.rhs(h, [])
    assert np.array_equal(np64(a[0]), np64(b[0]))
    assert all(np.array_equal(np64(x), np64(y)) for x, y in zip(a[1], b[1]))
    assert np.array_equal(np64(a[0]), np64(c[0]))
    # N commutes with every number-conserving generator: exactly zero
    assert np.all(np64(a[1][0]) == 0.0)


def test_rhs_four_operands_one_packed_block():
    """H and three observables: the largest set whose operands travel in one
    packed 32-byte block per index."""
    alg, nm, labels, h, xs = _case("mol5_3body")
    xs = xs + [np.random.default_rng(27).normal(size=len(labels))]
    G = graph_for("mol5_3body", alg, nm, labels)
    dh, dxs = G.rhs(h, xs)
    want_dh, want_dxs = oracle.rhs(alg, nm, labels, h, xs)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what="dh", atol=fl)
    for g_, w_ in zip(dxs, want_dxs):
        assert_close(np64(g_), w_, what="dx", atol=fl)


def test_rhs_many_operands_in_chunks():
    """More than four operands run as several record passes."""
    alg, nm, labels, h, _ = _case("mol5_3body")
    rng = np.random.default_rng(24)
    xs = [rng.normal(size=len(labels)) for _ in range(6)]
    G = graph_for("mol5_3body", alg, nm, labels)
    _, dxs = G.rhs(h, xs)
    _, want = oracle.rhs(alg, nm, labels, h, xs)
    for g_, w_ in zip(dxs, want):
        assert_close(np64(g_), w_)


def test_diagonal_only_registry_has_empty_generator_stage():
    labels = np.array([l for l in fermion_registry(4) if oracle.is_diagonal(ALG_FERMION, l)], dtype=np.uint64)
    G = graph_for("diag4", ALG_FERMION, 4, labels)
    assert G.R_g == 0 and G.R_L == 0
    dh, _ = G.rhs(np.arange(len(labels), dtype=np.float64) + 1.0)
    assert np.all(np64(dh) == 0.0)


@pytest.mark.parametrize("name", ["pauli3_ragged", "mol5_3body"])
def test_rhs_adjoint_matches_oracle(name):
    alg, nm, labels, h, xs = _case(name)
    G = graph_for(name, alg, nm, labels)
    rng = np.random.default_rng(25)
    wh = rng.normal(size=len(labels))
    wx = [rng.normal(size=len(labels)) for _ in xs]
    hb, xb = G.rhs_adjoint(h, xs, wh, wx)
    want_hb, want_xb = oracle.rhs_vjp(alg, nm, labels, h, xs, wh, wx)
    assert_close(np64(hb), want_hb, what="h_bar")
    for g_, w_ in zip(xb, want_xb):
        assert_close(np64(g_), w_, what="x_bar")


def test_rk4_flow_matches_oracle_closed_pauli():
    w = workload("closed_pauli_4q")
    rng = np.random.default_rng(26)
    x = rng.normal(size=len(w.labels))
    G = graph_for("pauli4", w.alg, w.nmodes, w.labels)
    nsteps = 40
    hs, xs, st, _ = G.flow(w.h, [x], method="rk4", s0=0.0, s1=nsteps * w.ds, ds=w.ds)
    assert st["steps"] == nsteps
    f = oracle.stacked_rhs(w.alg, w.nmodes, w.labels, 1)
    y = oracle.rk4_flow(f, np.concatenate([w.h, x]), w.ds, nsteps)
    assert_close(np64(hs), y[:len(w.labels)], what="h")
    assert_close(np64(xs[0]), y[len(w.labels):], what="x")


def test_rk4_full_flow_closed_pauli_equals_dense_wegner_flow():
    """Whole flow (ds = 1e-3 to s = 10): the closed-algebra coefficient flow
    is the 16x16 Wegner flow, step for step."""
    w = workload("closed_pauli_4q")
    G = graph_for("pauli4", w.alg, w.nmodes, w.labels)
    hs, _, st, _ = G.flow(w.h, [], method="rk4", s0=0.0, s1=w.s_end, ds=w.ds)
    assert st["steps"] == 10000
    H0 = dense.vec_matrix(w.labels, w.h, ALG_PAULI, 4)
    Hs = dense.rk4_dense(lambda B: dense.wegner_rhs(B)[0], H0, w.ds, 10000)
    assert_close(np64(hs), dense.pauli_coefficients(Hs, w.labels, 4).real, rtol=1e-9, what="h(s=10)")
    # Wegner flow drives the off-diagonal weight down
    od = np.array([not oracle.is_diagonal(ALG_PAULI, l) for l in w.labels])
    assert np.sum(np64(hs)[od] ** 2) < 1e-3 * np.sum(w.h[od] ** 2)


def test_dp45_flow_matches_oracle_replay_small_model():
    norb = 4
    labels = fermion_registry(norb)
    h = molecular_hamiltonian(labels, norb, seed=27, scale=0.2)
    xs = [number_operator(labels, norb), dipole_operator(labels, norb, seed=27)]
    G = graph_for("mol4", ALG_FERMION, norb, labels)
    hs, xo, st, steps = G.flow(h, xs, method="dp45", s0=0.0, s1=2.0, ds=1e-2, rtol=1e-10,
                               atol=1e-12)
    assert st["steps"] == len(steps) and abs(sum(steps) - 2.0) < 1e-12
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 2)
    y, _, _ = oracle.dp45_flow(f, np.concatenate([h] + xs), 0.0, 2.0, 1e-2, 1e-10, 1e-12, replay=steps)
    n = len(labels)
    assert_close(np64(hs), y[:n], what="h")
    assert_close(np64(xo[1]), y[2 * n:], what="dipole")
    # the free-running oracle takes (nearly) the same steps
    _, acc, rej = oracle.dp45_flow(f, np.concatenate([h] + xs), 0.0, 2.0, 1e-2, 1e-10, 1e-12)
    assert abs(len(acc) - st["steps"]) <= 2


def test_dp45_full_molecular_flow_equals_dense_sector_flows():
    """8 spin-orbitals, H + N + D, rtol 1e-10 to s = 10: the projected flow is
    the Wegner flow of the 8x8 (N=1) and 28x28 (N=2) blocks; replay the GPU's
    accepted steps on the blocks."""
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    hs, xo, st, steps = G.flow(w.h, w.observables, method="dp45", s0=0.0, s1=w.s_end, ds=w.ds,
                               rtol=w.rtol, atol=w.atol)
    assert st["steps"] > 10 and abs(sum(steps) - w.s_end) < 1e-9
    np.testing.assert_array_equal(np64(xo[0]), w.observables[0])      # N is carried unchanged
    A, B = oracle.DP_A[:6], oracle.DP_B[:6]
    for N in (1, 2):
        Hb = dense.sector_matrix(w.labels, w.h, 8, N)
        Db = dense.sector_matrix(w.labels, w.observables[1], 8, N)

        def f(Y):
            dB, eta = dense.wegner_rhs(Y[0])
            return np.stack([dB, eta @ Y[1] - Y[1] @ eta])

        Y = np.stack([Hb, Db])
        for ds in steps:
            Y = dense.rk_dense(f, Y, ds, A, B)
        assert_close(dense.sector_matrix(w.labels, np64(hs), 8, N), Y[0], rtol=1e-9, what=f"H block N={N}")
        assert_close(dense.sector_matrix(w.labels, np64(xo[1]), 8, N), Y[1], rtol=1e-9, what=f"D block N={N}")
        np.testing.assert_allclose(np.linalg.eigvalsh(Y[0]), np.linalg.eigvalsh(Hb), rtol=1e-8)


@pytest.mark.parametrize("method", ["rk4", "dp45"])
def test_flow_vjp_matches_oracle_discrete_adjoint(method):
    norb = 3
    labels = fermion_registry(norb)
    n = len(labels)
    h = molecular_hamiltonian(labels, norb, seed=28, scale=0.3)
    D = dipole_operator(labels, norb, seed=28)
    G = graph_for("mol3", ALG_FERMION, norb, labels)
    rng = np.random.default_rng(29)
    ybh, ybx = rng.normal(size=n), rng.normal(size=n)
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 1)
    fv = oracle.stacked_vjp(ALG_FERMION, norb, labels, 1)
    if method == "rk4":
        steps = [0.05] * 10
        gh, gx = G.flow_vjp(h, [D], ybh, [ybx], method="rk4", s0=0.0, s1=0.5, ds=0.05, checkpoint_every=3)
        _, want = oracle.rk_flow_vjp(f, fv, np.concatenate([h, D]), steps, oracle.RK4_A, oracle.RK4_B,
                                     np.concatenate([ybh, ybx]))
    else:
        _, _, _, steps = G.flow(h, [D], method="dp45", s0=0.0, s1=0.5, ds=0.02, rtol=1e-8, atol=1e-12)
        gh, gx = G.flow_vjp(h, [D], ybh, [ybx], method="dp45", s0=0.0, s1=0.5, steps=steps, checkpoint_every=4)
        _, want = oracle.rk_flow_vjp(f, fv, np.concatenate([h, D]), list(steps), oracle.DP_A[:6], oracle.DP_B[:6],
                                     np.concatenate([ybh, ybx]))
    assert_close(np64(gh), want[:n], what="grad h0")
    assert_close(np64(gx[0]), want[n:], what="grad x0")


def test_flow_reports_nonfinite_state():
    import paper_2609_14831_b300 as cg
    alg, nm, labels, h, xs = _case("mol5_3body")
    G = graph_for("mol5_3body", alg, nm, labels)
    bad = h.copy()
    bad[3] = np.nan
    with pytest.raises(cg.CutError) as e:
        G.flow(bad, [], method="rk4", s0=0.0, s1=0.01, ds=1e-3)
    assert e.value.name == "NONFINITE"
    with pytest.raises(cg.CutError) as e:
        G.flow(bad, [], method="dp45", s0=0.0, s1=0.01, ds=1e-3, rtol=1e-8)
    assert e.value.name == "NONFINITE"


def test_dp45_flow_pause_and_resume_is_exact():
    """Checkpoint/resume: a DP45 flow paused twice (after 100, then 150
    attempts) and resumed from (state, s_final, ds_next) takes the same
    accepted steps and ends on the same bits as the uninterrupted flow."""
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    kw = dict(method="dp45", s1=w.s_end, rtol=w.rtol, atol=w.atol)
    hs, xo, st, steps = G.flow(w.h, w.observables, s0=0.0, ds=w.ds, **kw)
    assert st["finished"] == 1
    h, x, s0, ds, got = w.h, list(w.observables), 0.0, w.ds, []
    for pause in (100, 150, 0):
        h, x, sti, stp = G.flow(h, x, s0=s0, ds=ds, pause_after=pause, **kw)
        got += list(stp)
        s0, ds = sti["s_final"], sti["ds_next"]
        assert sti["finished"] == (1 if pause == 0 else 0)
    np.testing.assert_array_equal(np.array(got), steps)
    np.testing.assert_array_equal(np64(h), np64(hs))
    for a, b in zip(x, xo):
        np.testing.assert_array_equal(np64(a), np64(b))

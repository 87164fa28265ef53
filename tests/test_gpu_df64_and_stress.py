"""Double-float arithmetic, the linear action L(h)x, and the full-size stress
graph (16 spin-orbitals, ~3.4e8 records) in the launch configuration the
benchmark times.

Full-size parity is checked on sparse inputs: the Hamiltonian and the
operands keep a seeded few hundred coefficients, so the oracle's exact
commutators stay cheap while the kernels still stream every record of the
real graph; the zero entries must come out exactly zero and every other
entry within RTOL of the oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_util import RTOL, assert_close, graph_for, np64, rhs_floor
from cut_inputs import (ALG_FERMION, cfg2_registry, dipole_operator, molecular_hamiltonian, number_operator,
                        workload)

pytestmark = pytest.mark.gpu


def _mol5():
    labels = cfg2_registry(5, keep_shared1=0.3, seed=3)
    h = molecular_hamiltonian(labels, 5, seed=22, scale=0.3)
    return labels, h, [number_operator(labels, 5), dipole_operator(labels, 5, seed=22)]


@pytest.mark.parametrize("name", ["mol8", "mol5_3body", "pauli4"])
def test_df64_rhs_matches_oracle(name):
    if name == "mol8":
        w = workload("molecular_8so")
        alg, nm, labels, h, xs = w.alg, w.nmodes, w.labels, w.h, w.observables
    elif name == "pauli4":
        w = workload("closed_pauli_4q")
        alg, nm, labels, h = w.alg, w.nmodes, w.labels, w.h
        xs = [np.random.default_rng(70).normal(size=len(labels))]
    else:
        labels, h, xs = _mol5()
        alg, nm = ALG_FERMION, 5
    G = graph_for(name + "_df", alg, nm, labels)
    G.set_arithmetic("df64")
    dh, dxs = G.rhs(h, xs)
    want_dh, want_dxs = oracle.rhs(alg, nm, labels, h, xs)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what="dh (df64)", atol=fl)
    for g_, w_ in zip(dxs, want_dxs):
        assert_close(np64(g_), w_, what="dx (df64)", atol=fl)


@pytest.mark.parametrize("n_obs", [3, 5])
def test_df64_rhs_with_operand_chunks(n_obs):
    """Double-float arithmetic takes up to three operands per pass over the
    records: four operands run as 3 + 1, six as 3 + 3."""
    labels, h, _ = _mol5()
    rng = np.random.default_rng(72 + n_obs)
    xs = [rng.normal(size=len(labels)) for _ in range(n_obs)]
    G = graph_for("mol5_3body_df", ALG_FERMION, 5, labels)
    G.set_arithmetic("df64")
    dh, dxs = G.rhs(h, xs)
    want_dh, want_dxs = oracle.rhs(ALG_FERMION, 5, labels, h, xs)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what="dh (df64)", atol=fl)
    assert len(dxs) == n_obs
    for g_, w_ in zip(dxs, want_dxs):
        assert_close(np64(g_), w_, what="dx (df64)", atol=fl)


def test_df64_flows_match_oracle():
    from cut_inputs import fermion_registry
    norb = 4
    labels = fermion_registry(norb)
    h = molecular_hamiltonian(labels, norb, seed=71, scale=0.2)
    xs = [number_operator(labels, norb), dipole_operator(labels, norb, seed=71)]
    G = graph_for("mol4_df", ALG_FERMION, norb, labels)
    G.set_arithmetic("df64")
    hs, xo, st, steps = G.flow(h, xs, method="dp45", s0=0.0, s1=1.0, ds=1e-2, rtol=1e-10, atol=1e-12)
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 2)
    y, _, _ = oracle.dp45_flow(f, np.concatenate([h] + xs), 0.0, 1.0, 1e-2, 1e-10, 1e-12, replay=steps)
    n = len(labels)
    assert_close(np64(hs), y[:n], what="h")
    assert_close(np64(xo[1]), y[2 * n:], what="D")
    hs4, _, _, _ = G.flow(h, xs, method="rk4", s0=0.0, s1=0.2, ds=0.02)
    y4 = oracle.rk4_flow(f, np.concatenate([h] + xs), 0.02, 10)
    assert_close(np64(hs4), y4[:n], what="h rk4")


def test_apply_L_is_the_commutator_stage():
    import torch
    labels, h, xs = _mol5()
    G = graph_for("mol5_3body", ALG_FERMION, 5, labels)
    dh, dxs, xi = G.rhs(h, xs, want_xi=True)
    rng = np.random.default_rng(72)
    extra = [rng.normal(size=len(labels)) for _ in range(5)]
    got = G.apply_L(xi, [h] + xs + extra)
    assert torch.equal(got[0], dh) and torch.equal(got[1], dxs[0]) and torch.equal(got[2], dxs[1])
    _, want = oracle.rhs(ALG_FERMION, 5, labels, h, extra)
    for g_, w_ in zip(got[3:], want):
        assert_close(np64(g_), w_, what="L(h) x")


def _sparse(v, keep, rng):
    out = np.zeros_like(v)
    idx = rng.choice(len(v), keep, replace=False)
    out[idx] = v[idx]
    return out


@pytest.fixture(scope="module")
def stress():
    w = workload("stress_16so")
    G = graph_for("stress16", w.alg, w.nmodes, w.labels)
    return w, G


def test_stress_graph_sizes_match_the_bench_table(stress):
    """The reference arm states the stress graph's sizes from a table."""
    import bench
    _, G = stress
    assert bench.GRAPH_SIZES["stress_16so"] == {"n": G.n, "n_g": G.n_g, "R_g": G.R_g, "R_L": G.R_L}


@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_stress_graph_full_size_sparse_input_parity(stress, arith):
    w, G = stress
    assert G.R_g + G.R_L > 3e8
    rng = np.random.default_rng(73)
    diag = np.array([int(l) & 0xFFFFFFFF == int(l) >> 32 for l in w.labels])
    h = _sparse(w.h, 200, rng)
    d_idx = np.nonzero(diag)[0]
    keep_d = rng.choice(d_idx, 40, replace=False)
    h[keep_d] = w.h[keep_d]
    xs = [_sparse(w.observables[1], 40, rng), _sparse(rng.normal(size=len(w.labels)), 150, rng)]
    G.set_arithmetic(arith)
    try:
        dh, dxs = G.rhs(h, xs)
    finally:
        G.set_arithmetic("fp64")
    want_dh, want_dxs = oracle.rhs(w.alg, w.nmodes, w.labels, h, xs)
    assert np.count_nonzero(want_dh) > 100
    for got, want in [(np64(dh), want_dh)] + [(np64(a), b) for a, b in zip(dxs, want_dxs)]:
        assert np.all(got[want == 0] == 0.0)
        assert_close(got, want, what=f"stress {arith}")


def test_stress_graph_full_size_properties(stress):
    """Dense seeded input at full size: the particle number commutes with
    every generator (its right-hand side is exactly zero), and the
    right-hand side of a Hermitian H is Hermitian: dh(C, A) = dh(A, C)."""
    w, G = stress
    dh, (dN, dD) = G.rhs(w.h, w.observables)
    assert np.all(np64(dN) == 0.0)
    dh = np64(dh)
    pos = {int(l): k for k, l in enumerate(w.labels)}
    mirror = np.array([pos[((int(l) & 0xFFFFFFFF) << 32) | (int(l) >> 32)] for l in w.labels])
    assert_close(dh[mirror], dh, rtol=1e-12, what="Hermiticity of dH")
    G.set_arithmetic("df64")
    try:
        dh2, _ = G.rhs(w.h, w.observables)
    finally:
        G.set_arithmetic("fp64")
    assert_close(np64(dh2), dh, rtol=1e-12, what="df64 vs fp64 at full size")


def test_outside_space_diagnostics_match_oracle():
    """C_q = coefficients of [eta, X] outside the registry (Eq. projected-flow),
    and the retained flow is the same with or without the diagnostic records."""
    from cut_inputs import fermion_registry
    from gpu_util import _TMP
    import os
    import paper_2609_14831_b300 as cg
    norb = 5
    labels = fermion_registry(norb)
    h = molecular_hamiltonian(labels, norb, seed=74, scale=0.3)
    xs = [dipole_operator(labels, norb, seed=74)]
    G = graph_for("mol5_plain", ALG_FERMION, norb, labels)
    path = os.path.join(_TMP, "mol5_diag.cutg")
    cg.build_graph(ALG_FERMION, norb, labels, path, diagnostics=True)
    Gd = cg.Graph(path, device=0)
    out_labels = Gd.outside_labels()
    C = Gd.rhs_outside(h, xs)
    for o, v in enumerate([h] + xs):
        full = oracle.rhs_unprojected(ALG_FERMION, norb, labels, h, v)
        want = np.array([complex(full.get(int(l), 0.0)).real for l in out_labels])
        # every generated term outside the registry has a row
        reg = {int(l) for l in labels}
        extra = {k for k, c in full.items() if abs(c) > 1e-13 and k not in reg} - {int(l) for l in out_labels}
        assert not extra
        assert_close(np64(C[o]), want, what=f"C operand {o}", atol=rhs_floor(h, xs))
    a = G.rhs(h, xs)
    b = Gd.rhs(h, xs)
    assert_close(np64(b[0]), np64(a[0]), rtol=1e-14, what="retained dh")
    fa = G.flow(h, xs, method="rk4", s0=0.0, s1=0.2, ds=0.02)
    fb = Gd.flow(h, xs, method="rk4", s0=0.0, s1=0.2, ds=0.02)
    assert_close(np64(fb[0]), np64(fa[0]), rtol=1e-13, what="retained flow")


def test_stress_graph_full_size_adjoint(stress):
    """The reverse traversal at full size (transposed record orders built at
    load, packed operand gathers, 8 lanes per row): the forward tangent and
    the vector-Jacobian product pair, <w, J v> = <J^T w, v>, and sampled
    operand adjoints x_bar_o[j] = <w_o, P[eta, O_j]> match the oracle on
    sparse inputs."""
    import paper_2609_14831_b300 as cg
    w, _ = stress
    G = cg.Graph(graph_for("stress16", w.alg, w.nmodes, w.labels).path, device=0, adjoint=True)
    rng = np.random.default_rng(75)
    n = len(w.labels)
    h, xs = w.h, list(w.observables)
    v_h, v_x = rng.normal(size=n), [rng.normal(size=n) for _ in xs]
    w_h, w_x = rng.normal(size=n), [rng.normal(size=n) for _ in xs]
    jh, jx = G.rhs_jvp(h, xs, v_h, v_x)
    bh, bx = G.rhs_adjoint(h, xs, w_h, w_x)
    lhs = w_h @ np64(jh) + sum(a @ np64(b) for a, b in zip(w_x, jx))
    rhs = np64(bh) @ v_h + sum(np64(a) @ b for a, b in zip(bx, v_x))
    scale = np.abs(w_h) @ np.abs(np64(jh)) + sum(np.abs(a) @ np.abs(np64(b)) for a, b in zip(w_x, jx))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    # sampled operand adjoints on sparse inputs against the oracle
    hs = _sparse(w.h, 300, rng)
    diag = np.nonzero([int(l) & 0xFFFFFFFF == int(l) >> 32 for l in w.labels])[0]
    keep = rng.choice(diag, 40, replace=False)
    hs[keep] = w.h[keep]
    ws = [_sparse(rng.normal(size=n), 2000, rng) for _ in range(3)]
    bh, bx = G.rhs_adjoint(hs, xs, ws[0], ws[1:])
    eta = oracle.generator(w.alg, w.nmodes, w.labels, hs)
    for j in rng.choice(n, 12, replace=False):
        col = oracle.project(oracle.commutator(w.alg, w.nmodes, eta, {int(w.labels[j]): 1.0}), w.labels).real
        for o, got in enumerate([None] + list(bx)):
            if o == 0:
                continue
            want = col @ ws[o]
            assert abs(np64(got)[j] - want) <= 1e-10 * (abs(want) + np.abs(col) @ np.abs(ws[o])) + 1e-300, (j, o)
    G.close()


@pytest.mark.parametrize("n_obs", [4, 7, 8])
def test_packed_adjoint_operand_counts_match_oracle(n_obs):
    """Five and eight operands (one and a part, and two full packed blocks) in
    the packed transposed passes; nine operands take the unpacked kernels."""
    from cut_inputs import fermion_registry
    labels = fermion_registry(4)
    h = molecular_hamiltonian(labels, 4, seed=76, scale=0.3)
    rng = np.random.default_rng(76 + n_obs)
    xs = [rng.normal(size=len(labels)) for _ in range(n_obs)]
    G = graph_for("mol4", ALG_FERMION, 4, labels)
    wh = rng.normal(size=len(labels))
    wx = [rng.normal(size=len(labels)) for _ in xs]
    hb, xb = G.rhs_adjoint(h, xs, wh, wx)
    want_hb, want_xb = oracle.rhs_vjp(ALG_FERMION, 4, labels, h, xs, wh, wx)
    assert_close(np64(hb), want_hb, what="h_bar")
    for g_, w_ in zip(xb, want_xb):
        assert_close(np64(g_), w_, what="x_bar")


@pytest.mark.parametrize("arith,n_obs", [("fp64", 1), ("fp64", 4), ("df64", 2)])
def test_few_long_rows_cut_into_pieces_match_oracle(arith, n_obs):
    """The closed 6-qubit Pauli registry has 4,096 rows of 2,016 records
    each, few and long, so the commutator stage cuts every row into pieces
    of about 256 records and adds each row's pieces in order.  Against the
    oracle (FP64 and double-float, one to five operands), repeatable bit for
    bit, and equal within the parity tolerance to the allocation-free entry
    point, which sums whole rows."""
    import ctypes
    import torch
    import paper_2609_14831_b300 as cg
    from cut_inputs import ALG_PAULI, pauli_registry
    labels = pauli_registry(6)
    rng = np.random.default_rng(77 + n_obs)
    h = rng.normal(size=len(labels)) * 0.1
    xs = [rng.normal(size=len(labels)) for _ in range(n_obs)]
    G = graph_for("pauli6", ALG_PAULI, 6, labels)
    G.set_arithmetic(arith)
    try:
        dh, dxs = G.rhs(h, xs)
        dh2, dxs2 = G.rhs(h, xs)
    finally:
        G.set_arithmetic("fp64")
    assert torch.equal(dh, dh2) and all(torch.equal(a, b) for a, b in zip(dxs, dxs2))
    want_dh, want_dxs = oracle.rhs(ALG_PAULI, 6, labels, h, xs)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what=f"dh ({arith})", atol=fl)
    for g_, w_ in zip(dxs, want_dxs):
        assert_close(np64(g_), w_, what=f"dx ({arith})", atol=fl)
    if arith == "fp64":
        hd = torch.tensor(h, device="cuda")
        X = torch.tensor(np.stack(xs), device="cuda")
        oh, oX = torch.empty_like(hd), torch.empty_like(X)
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        cg.check(cg.lib().cut_rhs_noalloc(G._h, P(hd), n_obs, P(X), P(oh), P(oX),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        assert_close(np64(oh), np64(dh), what="whole rows vs pieces", atol=fl)

"""Batched flows (many parameter sets, one graph read per record) on the GPU.

FP64 batched RK4 must match the oracle's RK4 flow of every instance at
RTOL = 1e-10.  FP64 batched DP45 takes each instance's own adaptive path and
is compared with the single-instance GPU flow (same controller) and its step
count.  The FP32-record path is compared with FP64 and its error reported.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_util import assert_close, graph_for, np64
from cut_inputs import (ALG_FERMION, batched_parameters, dipole_operator, fermion_registry,
                        number_operator, workload, cfg2_registry, molecular_hamiltonian)

pytestmark = pytest.mark.gpu


def _batch(norb, B, seed):
    labels = fermion_registry(norb)
    H = batched_parameters(labels, norb, B, seed=seed)
    N = number_operator(labels, norb)
    D = dipole_operator(labels, norb, seed=seed)
    X = np.stack([np.stack([N, D])] * B)
    return labels, H, X


@pytest.mark.parametrize("tile", [0, 2, 8])
def test_batched_rk4_fp64_matches_oracle(tile):
    import torch
    norb, B = 4, 37                       # ragged against every tile width
    labels, H, X = _batch(norb, B, seed=31)
    G = graph_for("mol4", ALG_FERMION, norb, labels)
    Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="rk4",
                                           s0=0.0, s1=0.2, ds=0.02, tile=tile)
    assert np.all(status.cpu().numpy() == 0) and np.all(steps.cpu().numpy() == 10)
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, 2)
    n = len(labels)
    for b in (0, 5, 17, 36):
        y = oracle.rk4_flow(f, np.concatenate([H[b], X[b, 0], X[b, 1]]), 0.02, 10)
        assert_close(np64(Hs[b]), y[:n], what=f"h[{b}]")
        assert_close(np64(Xs[b, 1]), y[2 * n:], what=f"D[{b}]")


def test_batched_dp45_fp64_follows_single_instance_flows():
    import torch
    w = workload("molecular_8so")
    B = 24
    H = batched_parameters(w.labels, 8, B, seed=32)
    X = np.stack([np.stack(w.observables)] * B)
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="dp45",
                                           s0=0.0, s1=2.0, ds=1e-2, rtol=1e-10, atol=1e-12)
    steps = steps.cpu().numpy()
    assert np.all(status.cpu().numpy() == 0)
    assert len(set(steps.tolist())) > 1          # uneven step counts across the batch
    for b in (0, 7, 23):
        hs, xs, st, _ = G.flow(H[b], list(X[b]), method="dp45", s0=0.0, s1=2.0, ds=1e-2, rtol=1e-10, atol=1e-12)
        assert abs(st["steps"] - steps[b]) <= 2
        # same tolerance-controlled path: agreement at the integration tolerance
        assert_close(np64(Hs[b]), np64(hs), rtol=1e-8, what=f"h[{b}]")
        assert_close(np64(Xs[b, 1]), np64(xs[1]), rtol=1e-8, what=f"D[{b}]")


def test_batched_fp32_records_error_against_fp64():
    import torch
    w = workload("molecular_8so")
    B = 64
    H = batched_parameters(w.labels, 8, B, seed=33)
    X = np.stack([np.stack(w.observables)] * B)
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    H64, X64, st64, _ = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="dp45",
                                       s0=0.0, s1=10.0, ds=1e-2, rtol=1e-10, atol=1e-12)
    H32, X32, st32, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp32", method="dp45",
                                            s0=0.0, s1=10.0, ds=1e-2, rtol=1e-6, atol=1e-9)
    assert np.all(status.cpu().numpy() == 0)
    err = np.max(np.abs(np64(H32) - np64(H64)), axis=1) / np.max(np.abs(np64(H64)), axis=1)
    print(f"FP32-record batched flow vs FP64: max rel error {err.max():.2e}, median {np.median(err):.2e}")
    assert err.max() < 1e-4
    assert np.all(np64(X32[:, 0]) == np64(X64[:, 0]))     # N is exactly conserved in both


def test_batched_rejects_bad_arguments():
    import torch
    import paper_2609_14831_b300 as cg
    labels, H, X = _batch(4, 3, seed=34)
    G = graph_for("mol4", ALG_FERMION, 4, labels)
    with pytest.raises(cg.CutError):
        G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="rk4", s0=0.0, s1=0.1, ds=0.01, tile=3)


def test_batched_refills_slots_and_matches_single_instance_flows():
    """More instances than resident slots (1500 > 148 CTAs x 8 slots): slots
    that finish are refilled from the queue inside the kernel.  Every
    instance, first wave or refilled, equals its own single-instance FP64
    flow; the FP32-record batch stays within its stated error."""
    import torch
    w = workload("molecular_8so")
    B = 1500
    H = batched_parameters(w.labels, 8, B, seed=35)
    X = np.stack([np.stack(w.observables)] * B)
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    kw = dict(method="rk4", s0=0.0, s1=0.02, ds=0.01, tile=8)
    Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", **kw)
    assert np.all(status.cpu().numpy() == 0) and np.all(steps.cpu().numpy() == 2)
    for b in (0, 1, 1035, 1183, 1184, 1499):
        hs, xs, st, _ = G.flow(H[b], list(X[b]), method="rk4", s0=0.0, s1=0.02, ds=0.01)
        assert st["steps"] == 2
        assert_close(np64(Hs[b]), np64(hs), what=f"h[{b}]")
        assert_close(np64(Xs[b, 1]), np64(xs[1]), what=f"D[{b}]")
    H32, X32, _, status32 = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp32", **kw)
    assert np.all(status32.cpu().numpy() == 0)
    err = np.max(np.abs(np64(H32) - np64(Hs)), axis=1) / np.max(np.abs(np64(Hs)), axis=1)
    assert err.max() < 1e-5, err.max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_single_instance(precision):
    import torch
    labels, H, X = _batch(4, 1, seed=36)
    G = graph_for("mol4", ALG_FERMION, 4, labels)
    tol = dict(rtol=1e-10, atol=1e-12) if precision == "fp64" else dict(rtol=1e-6, atol=1e-9)
    Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision=precision, method="dp45",
                                           s0=0.0, s1=1.0, ds=1e-2, **tol)
    assert int(status[0]) == 0
    hs, xs, st, _ = G.flow(H[0], list(X[0]), method="dp45", s0=0.0, s1=1.0, ds=1e-2, rtol=1e-10, atol=1e-12)
    assert_close(np64(Hs[0]), np64(hs), rtol=1e-8 if precision == "fp64" else 1e-4, what="h")


def test_batched_diagonal_only_registry_is_stationary():
    """No generator and no commutator records: every instance keeps its
    coefficients bit for bit (the empty stages write exact zeros)."""
    import torch
    labels = np.array([l for l in fermion_registry(4) if oracle.is_diagonal(ALG_FERMION, l)], dtype=np.uint64)
    G = graph_for("diag4", ALG_FERMION, 4, labels)
    rng = np.random.default_rng(37)
    H = rng.normal(size=(9, len(labels)))
    X = rng.normal(size=(9, 1, len(labels)))
    for precision in ("fp64", "fp32"):
        Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision=precision, method="rk4",
                                               s0=0.0, s1=0.1, ds=0.05)
        assert np.all(status.cpu().numpy() == 0)
        np.testing.assert_array_equal(np64(Hs), H)
        np.testing.assert_array_equal(np64(Xs), X)


@pytest.mark.parametrize("n_obs", [0, 3])
def test_batched_rk4_fp64_operand_counts(n_obs):
    """No observable (H alone) and three observables (four operands, the
    most a batch carries) against the oracle's RK4 flow."""
    import torch
    norb, B = 4, 11
    labels = fermion_registry(norb)
    H = batched_parameters(labels, norb, B, seed=38)
    rng = np.random.default_rng(38)
    obs = [number_operator(labels, norb), dipole_operator(labels, norb, seed=38), rng.normal(size=len(labels))]
    X = np.stack([np.stack(obs[:n_obs])] * B) if n_obs else None
    G = graph_for("mol4", ALG_FERMION, norb, labels)
    Hs, Xs, steps, status = G.flow_batched(torch.tensor(H), None if X is None else torch.tensor(X),
                                           precision="fp64", method="rk4", s0=0.0, s1=0.1, ds=0.02, tile=4)
    assert np.all(status.cpu().numpy() == 0) and np.all(steps.cpu().numpy() == 5)
    f = oracle.stacked_rhs(ALG_FERMION, norb, labels, n_obs)
    n = len(labels)
    for b in (0, 6, 10):
        y = oracle.rk4_flow(f, np.concatenate([H[b]] + [X[b, o] for o in range(n_obs)]), 0.02, 5)
        assert_close(np64(Hs[b]), y[:n], what=f"h[{b}]")
        for o in range(n_obs):
            assert_close(np64(Xs[b, o]), y[(o + 1) * n:(o + 2) * n], what=f"x{o}[{b}]")


@pytest.mark.parametrize("n_obs", [1, 3])
def test_batched_fp32_operand_layouts(n_obs):
    """FP32 records with two operands (pairs) and four (the padded block's
    full width) against the FP64 batch of the same flows."""
    import torch
    norb, B = 4, 19
    labels = fermion_registry(norb)
    H = batched_parameters(labels, norb, B, seed=39)
    rng = np.random.default_rng(39)
    obs = [dipole_operator(labels, norb, seed=39), number_operator(labels, norb), rng.normal(size=len(labels))]
    X = torch.tensor(np.stack([np.stack(obs[:n_obs])] * B))
    G = graph_for("mol4", ALG_FERMION, norb, labels)
    kw = dict(method="rk4", s0=0.0, s1=0.2, ds=0.02)
    H64, X64, _, st64 = G.flow_batched(torch.tensor(H), X, precision="fp64", **kw)
    H32, X32, _, st32 = G.flow_batched(torch.tensor(H), X, precision="fp32", **kw)
    assert np.all(st64.cpu().numpy() == 0) and np.all(st32.cpu().numpy() == 0)
    for a, b in ((H32, H64), (X32, X64)):
        a, b = np64(a), np64(b)
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err < 1e-5, err


def _sector_replay(labels, h0, D0, steps, N):
    """Dense Wegner flow of the N-particle block of (H, D) along the given
    accepted Dormand-Prince steps (the oracle's tableau).  Rank-3 terms
    annihilate every state with at most two particles, so the projected
    flow of the <=2-body registry is this flow exactly (pinned on CPU by
    test_oracle_pins.test_fermion_flow_matches_sector_wegner_flows)."""
    import dense
    A, B = oracle.DP_A[:6], oracle.DP_B[:6]

    def f(Y):
        dB, eta = dense.wegner_rhs(Y[0])
        return np.stack([dB, eta @ Y[1] - Y[1] @ eta])
    Y = np.stack([dense.sector_matrix(labels, h0, 8, N), dense.sector_matrix(labels, D0, 8, N)])
    for ds in steps:
        Y = dense.rk_dense(f, Y, ds, A, B)
    return Y


def test_batched_full_size_dp45_matches_oracle_replay():
    """The benchmarked batch itself: 8 spin-orbitals, 1024 parameter sets,
    H + N + D, DP45 rtol 1e-10 to s = 10, FP64.  Four instances spread over
    the batch replay their own recorded accepted steps in the oracle's
    Dormand-Prince tableau on the dense N=1 and N=2 blocks, and must agree
    element by element at 1e-10 of the block's largest entry.  Over a short
    span one instance of the same batch is also replayed through the
    string-algebra oracle itself.  The FP32-record batch (rtol 1e-6) is then compared with
    this FP64 batch instance by instance; its error is stated per result."""
    import torch
    import dense
    w = workload("molecular_8so")
    B = 1024
    H = batched_parameters(w.labels, 8, B, seed=3)
    X = np.stack([np.stack(w.observables)] * B)
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    H64, X64, st64, status, rec = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64",
                                                 method="dp45", s0=0.0, s1=10.0, ds=1e-2, rtol=1e-10,
                                                 atol=w.atol, record_cap=4096)
    st64, rec = st64.cpu().numpy(), np64(rec)
    assert np.all(status.cpu().numpy() == 0)
    assert st64.max() < 4096 and len(set(st64.tolist())) > 1
    for b in (0, 341, 682, 1023):
        steps = rec[b, :st64[b]]
        assert np.all(steps > 0) and np.all(rec[b, st64[b]:] == 0)
        assert abs(steps.sum() - 10.0) < 1e-9, steps.sum()
        np.testing.assert_array_equal(np64(X64[b, 0]), w.observables[0])     # N is carried unchanged
        for N in (1, 2):
            Y = _sector_replay(w.labels, H[b], w.observables[1], steps, N)
            assert_close(dense.sector_matrix(w.labels, np64(H64[b]), 8, N), Y[0], rtol=1e-10,
                         what=f"instance {b} H block N={N}")
            assert_close(dense.sector_matrix(w.labels, np64(X64[b, 1]), 8, N), Y[1], rtol=1e-10,
                         what=f"instance {b} D block N={N}")
    # the string-algebra oracle itself, along the steps that instance 682 of
    # the same 1024-instance batch takes over a short span (s in [0, 0.01])
    b = 682
    Hs, Xs, sts, status2, recs = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64",
                                                method="dp45", s0=0.0, s1=0.01, ds=5e-3, rtol=1e-10,
                                                atol=w.atol, record_cap=16)
    assert np.all(status2.cpu().numpy() == 0)
    steps = list(np64(recs)[b, :int(sts[b])])
    assert 1 <= len(steps) <= 6 and abs(sum(steps) - 0.01) < 1e-15
    f = oracle.stacked_rhs(w.alg, w.nmodes, w.labels, 2)
    y, _, _ = oracle.dp45_flow(f, np.concatenate([H[b], X[b, 0], X[b, 1]]), 0.0, 0.01, 5e-3, 1e-10, w.atol,
                               replay=steps)
    n = len(w.labels)
    assert_close(np64(Hs[b]), y[:n], what="batched h vs oracle replay")
    assert_close(np64(Xs[b, 1]), y[2 * n:], what="batched D vs oracle replay")
    # FP32 records against the FP64 batch, per instance
    H32, X32, st32, status32 = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp32", method="dp45",
                                              s0=0.0, s1=10.0, ds=1e-2, rtol=1e-6, atol=1e-9)
    assert np.all(status32.cpu().numpy() == 0)
    a, r = np64(H32), np64(H64)
    err = np.max(np.abs(a - r), axis=1) / np.max(np.abs(r), axis=1)
    print(f"FP32-record batch vs oracle-checked FP64 batch, per instance (1024): median {np.median(err):.2e}, "
          f"p99 {np.percentile(err, 99):.2e}, max {err.max():.2e}")
    assert err.max() < 1e-4


def test_tile_choices_persist_in_the_tune_cache_file(tmp_path):
    """CUT_TUNE_CACHE: the autotuner appends its choice (graph SHA-256,
    batch, operands, precision, method, tile, GPU name) and a later lookup
    takes a remembered width from a file instead of probing.  Every width
    sums each instance in record order, so the width changes no bits."""
    import torch
    w = workload("molecular_4so")
    G = graph_for("mol4_workload", w.alg, w.nmodes, w.labels)
    B = 29                                  # a batch size no other test tunes
    H = torch.tensor(batched_parameters(w.labels, 4, B, seed=77))
    X = torch.tensor(np.stack([np.stack(w.observables)] * B))
    first = tmp_path / "tune1.txt"
    os.environ["CUT_TUNE_CACHE"] = str(first)
    try:
        Ha, Xa, sa, sta = G.flow_batched(H, X, precision="fp64", method="dp45", s0=0.0, s1=0.5, ds=1e-2,
                                         rtol=1e-8, atol=1e-12)
        tuned = G.last_batched_tile()
        lines = first.read_text().splitlines()
        assert len(lines) == 1
        sha, batch, nops, fp32, method, tile, *name = lines[0].split()
        assert (int(batch), int(nops), int(fp32), int(tile)) == (B, 1 + len(w.observables), 0, tuned)
        assert len(sha) == 64 and name
        # a second file remembers another width for the same key
        other = 4 if tuned != 4 else 2
        second = tmp_path / "tune2.txt"
        second.write_text(" ".join([sha, batch, nops, fp32, method, str(other)] + name) + "\n")
        os.environ["CUT_TUNE_CACHE"] = str(second)
        Hb, Xb, sb, stb = G.flow_batched(H, X, precision="fp64", method="dp45", s0=0.0, s1=0.5, ds=1e-2,
                                         rtol=1e-8, atol=1e-12)
        assert G.last_batched_tile() == other
        assert second.read_text().count("\n") == 1      # nothing probed, nothing appended
        np.testing.assert_array_equal(np64(Hb), np64(Ha))
        np.testing.assert_array_equal(np64(sb), np64(sa))
    finally:
        os.environ.pop("CUT_TUNE_CACHE", None)

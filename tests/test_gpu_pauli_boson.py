"""Pauli-boson graphs on the GPU (the paper's algebra, Sec. 2.1).

The stored factors here take many magnitudes (normal-ordering integers), so
these graphs run the general factor path of the kernels.  Right-hand sides
against the oracle at RTOL (two-mode registry dense; the five-mode
7,017,036-record graph on a sparse input), an eight-operand action, and a
short RK4 flow against the oracle's flow.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close, graph_for, np64, rhs_floor
from cut_inputs import ALG_PAULI_BOSON, pauli_boson_hamiltonian, pauli_boson_registry

pytestmark = pytest.mark.gpu


def test_two_mode_rhs_and_flow_match_oracle():
    M, p = 2, 4
    labels = pauli_boson_registry(M, p)
    h = pauli_boson_hamiltonian(labels, M, seed=91)
    xs = [pauli_boson_hamiltonian(labels, M, seed=92 + i) for i in range(7)]   # 8 operands, one record pass
    G = graph_for("pb2m4", ALG_PAULI_BOSON, M, labels)
    dh, dxs = G.rhs(h, xs)
    want_dh, want_dxs = oracle.rhs(ALG_PAULI_BOSON, M, labels, h, xs)
    fl = rhs_floor(h, xs)
    assert_close(np64(dh), want_dh, what="dh", atol=fl)
    for g_, w_ in zip(dxs, want_dxs):
        assert_close(np64(g_), w_, what="dx (8-operand block)", atol=fl)
    hs, _, _, _ = G.flow(h, xs[:1], method="rk4", s0=0.0, s1=0.05, ds=0.01)
    f = oracle.stacked_rhs(ALG_PAULI_BOSON, M, labels, 1)
    y = oracle.rk4_flow(f, np.concatenate([h, xs[0]]), 0.01, 5)
    assert_close(np64(hs), y[:len(labels)], what="flowed h")


def test_five_mode_graph_sparse_input_parity():
    M, p = 5, 4
    labels = pauli_boson_registry(M, p)
    G = graph_for("pb5m4", ALG_PAULI_BOSON, M, labels)
    assert G.R_g + G.R_L == 7017036
    full = pauli_boson_hamiltonian(labels, M, seed=93)
    rng = np.random.default_rng(94)
    keep = rng.choice(len(labels), 250, replace=False)
    diag = np.nonzero([oracle.is_diagonal(ALG_PAULI_BOSON, l) for l in labels])[0]
    h = np.zeros_like(full)
    h[keep] = full[keep]
    h[diag] = full[diag]
    x = np.zeros_like(full)
    x[keep[:100]] = rng.normal(size=100)
    dh, (dx,) = G.rhs(h, [x])
    want_dh, (want_dx,) = oracle.rhs(ALG_PAULI_BOSON, M, labels, h, [x])
    fl = rhs_floor(h, [x])
    assert_close(np64(dh), want_dh, what="dh", atol=fl)
    assert_close(np64(dx), want_dx, what="dx", atol=fl)

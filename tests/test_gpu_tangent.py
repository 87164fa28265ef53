"""Forward tangent (directional derivative, Sec. 2.4) on the GPU.

Against the oracle's exact tangent (five-point formula on the cubic
right-hand side) at RTOL, and the paper's validation pattern: centred finite
differences of the GPU right-hand side over eps = 1e-3 .. 1e-5 for
perturbations of the Hamiltonian (including the generator variation) and of
the operand, maximum relative error small over that window.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close, graph_for, np64, rhs_floor
from cut_inputs import ALG_FERMION, ALG_PAULI, cfg2_registry, dipole_operator, molecular_hamiltonian, pauli_registry

pytestmark = pytest.mark.gpu


def _mol5():
    labels = cfg2_registry(5, keep_shared1=0.3, seed=3)
    h = molecular_hamiltonian(labels, 5, seed=22, scale=0.3)
    return ALG_FERMION, 5, labels, h, [dipole_operator(labels, 5, seed=22)]


@pytest.mark.parametrize("case", ["mol5_3body", "pauli3"])
def test_jvp_matches_oracle_tangent(case):
    if case == "pauli3":
        labels = pauli_registry(3)
        rng0 = np.random.default_rng(80)
        alg, nm, h, xs = ALG_PAULI, 3, rng0.normal(size=len(labels)), [rng0.normal(size=len(labels))]
    else:
        alg, nm, labels, h, xs = _mol5()
    G = graph_for(case if case != "pauli3" else "pauli3_full", alg, nm, labels)
    rng = np.random.default_rng(81)
    dh = rng.normal(size=len(labels)) * 0.1
    dxs = [rng.normal(size=len(labels)) for _ in xs]
    gh, gx = G.rhs_jvp(h, xs, dh, dxs)
    wh, wx = oracle.rhs_jvp(alg, nm, labels, h, xs, dh, dxs)
    fl = rhs_floor(h, xs)
    assert_close(np64(gh), wh, what="tangent h", atol=fl)
    assert_close(np64(gx[0]), wx[0], what="tangent x", atol=fl)


def test_jvp_against_centred_differences_scan():
    alg, nm, labels, h, xs = _mol5()
    G = graph_for("mol5_3body", alg, nm, labels)
    rng = np.random.default_rng(82)
    # directions of 1% of the coefficient scale: the central-difference
    # truncation error ~ (eps |d|)^2 stays below the rounding error over the
    # whole window, as in the paper's validation window
    hs, xsc = np.max(np.abs(h)), np.max(np.abs(xs[0]))
    for which in ("h", "x"):
        dh = 1e-2 * hs * rng.normal(size=len(labels)) if which == "h" else np.zeros(len(labels))
        dx = 1e-2 * xsc * rng.normal(size=len(labels)) if which == "x" else np.zeros(len(labels))
        jh, jx = G.rhs_jvp(h, xs, dh, [dx])
        j = np.concatenate([np64(jh), np64(jx[0])])
        worst = 0.0
        for eps in (1e-3, 3e-4, 1e-4, 3e-5, 1e-5):
            p = G.rhs(h + eps * dh, [xs[0] + eps * dx])
            m = G.rhs(h - eps * dh, [xs[0] - eps * dx])
            fd = (np.concatenate([np64(p[0]), np64(p[1][0])]) - np.concatenate([np64(m[0]), np64(m[1][0])])) / (2 * eps)
            worst = max(worst, np.max(np.abs(fd - j)) / np.max(np.abs(j)))
        print(f"tangent vs centred differences ({which}): max relative error {worst:.2e}")
        assert worst < 1e-8

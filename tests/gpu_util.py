"""Shared helpers of the GPU tests (no oracle arithmetic here)."""
import os
import tempfile

import numpy as np

import paper_2609_14831_b300 as cg

_CACHE = {}
_TMP = tempfile.mkdtemp(prefix="cutg_tests_")

# Parity tolerance for FP64 coefficients: every element within
# RTOL * (|want| + max|want|); the graph reproduces the oracle's finite
# algebra exactly, so only summation order differs (about 1e-15 relative).
RTOL = 1e-10


def rhs_floor(h, xs=()):
    """Absolute floor for right-hand-side comparisons: the terms of
    P[eta, X] are products xi * x with |xi| <= O(|h|^2), so both sides carry
    rounding of about 1e-16 of max|h|^2 max|x| times the number of terms.
    A vector whose exact value is zero (e.g. the particle number, which
    commutes with every generator) is compared against this floor."""
    hm = float(np.max(np.abs(h)))
    xm = max([hm] + [float(np.max(np.abs(x))) for x in xs])
    return 1e-12 * hm * hm * xm


def assert_close(got, want, rtol=RTOL, what="", atol=0.0):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (got.shape, want.shape)
    scale = float(np.max(np.abs(want))) if want.size else 0.0
    err = np.abs(got - want)
    lim = rtol * (np.abs(want) + scale) + atol + 1e-300
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, f"{what}: {bad.size} elements off, worst {err.max():.3e} (scale {scale:.3e}) at {bad[:5]}"


def graph_for(key, alg, nmodes, labels, **kw):
    """Build once per test session and load on cuda:0."""
    if key not in _CACHE:
        path = os.path.join(_TMP, f"{key}.cutg")
        cg.build_graph(alg, nmodes, labels, path, **kw)
        _CACHE[key] = cg.Graph(path, device=0)
    return _CACHE[key]


def np64(t):
    return t.detach().cpu().numpy().astype(np.float64)

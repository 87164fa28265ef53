"""The learned surrogate: trained by the library's own kernels on flows the
batched path generates; checked for what it gains over the plain flow.

Small-scale version of the surrogate workload (the benchmark runs the full
one): 8-spin-orbital model, 32 parameters theta ~ U(-0.1, 0.1) about the
reference Hamiltonian, training set from FP32-record batched flows.  The
screened quantities are the 36 diagonal coefficients; the gate is 1e-4.
"""
import numpy as np
import pytest

from gpu_util import graph_for
from cut_inputs import parameter_directions, workload

pytestmark = pytest.mark.gpu


def test_surrogate_gain_with_plain_flow_fallback():
    import torch
    from paper_2609_14831_b300.surrogate import Surrogate
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    P = parameter_directions(w.labels, 8)
    sur = Surrogate(G, w.h, P, w.observables, n_hidden=512, seed=0)
    rng = np.random.default_rng(50)
    th_train = rng.uniform(-0.1, 0.1, size=(4096, 32))
    th_test = rng.uniform(-0.1, 0.1, size=(256, 32))
    Htr, steps = sur.flows(th_train, "fp32")
    assert len(set(steps.cpu().numpy().tolist())) > 1
    hist = sur.fit(th_train, Htr, epochs=300, batch=256, lr=3e-3)
    print(f"training loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert hist[-1] < 0.1 * hist[0]
    diag = np.nonzero([int(l) & 0xFFFFFFFF == int(l) >> 32 for l in w.labels])[0]
    assert len(diag) == 36
    exact, _ = sur.flows(th_test, "fp64")
    pred = sur.predict(th_test)
    err_net = (pred[:, diag] - exact[:, diag]).abs().max(dim=1).values.cpu().numpy()
    out, ok, tm = sur.screen(th_test, diag, tol=1e-4)
    ok = ok.cpu().numpy()
    err = (out[:, diag] - exact[:, diag]).abs().max(dim=1).values.cpu().numpy()
    print(f"surrogate: accepted {ok.sum()}/{len(ok)}, median net error {np.median(err_net):.2e}, "
          f"max error of accepted {err[ok].max() if ok.any() else 0:.2e}, timings {tm}")
    # every answer is within the gate (plus the loose flow's own error) of the FP64 flow
    assert np.all(err <= 1e-4 + 1e-5)
    # rejected queries get the FP64 flow (another batch composition may pick
    # another tile width, so agreement is at the flow tolerance)
    if (~ok).any():
        assert np.all(err[~ok] <= 1e-8)
    # the network resolves a share of the queries without the FP64 flow
    assert ok.mean() > 0.2

"""The learned surrogate: trained by the library's own kernels on flows the
batched path generates; checked for what it gains over the plain flow.

Small-scale version of the surrogate workload (the benchmark's --surrogate
mode runs the 50k-flow one): 8-spin-orbital model, 32 parameters
theta ~ U(-0.1, 0.1) about the reference Hamiltonian, training set from
FP32-record batched flows, held-out queries checked against FP64 flows.

Two uses are measured:
  * screen: find the 10% of queries with the lowest flowed coefficient of n_0
    (the lowest orbital) by ranking the network's predictions and running the
    FP64 flow only on the best-ranked 30%; the gain is the FP64 flows avoided
    at the measured recall;
  * gate: answers whose prediction of the lowest diagonal coefficient (n_0,
    the quantity the gradient workload targets) is within 1e-4 of a loose
    FP32 flow are served by the network, the rest by the FP64 flow -- every
    answer must then be within the gate of the FP64 flow.  The same gate on
    all 36 diagonal coefficients is reported (the two-particle diagonals
    vary roughly with theta near the degenerate pair energies).
"""
import numpy as np
import pytest

from gpu_util import graph_for
from cut_inputs import make_label, parameter_directions, workload

pytestmark = pytest.mark.gpu


def test_surrogate_screen_and_gate():
    from paper_2609_14831_b300.surrogate import Surrogate
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    P = parameter_directions(w.labels, 8)
    sur = Surrogate(G, w.h, P, w.observables, n_hidden=512, seed=0)
    rng = np.random.default_rng(50)
    th_train = rng.uniform(-0.1, 0.1, size=(4096, 32))
    th_test = rng.uniform(-0.1, 0.1, size=(512, 32))
    Htr, steps = sur.flows(th_train, "fp32")
    assert len(set(steps.cpu().numpy().tolist())) > 1
    hist = sur.fit(th_train, Htr, epochs=200, batch=256, lr=3e-3)
    print(f"training loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    assert hist[-1] < 0.2 * hist[0]
    k0 = int(np.nonzero(w.labels == np.uint64(make_label(1, 1)))[0][0])
    exact, _ = sur.flows(th_test, "fp64")
    pred = sur.predict(th_test)
    e_true = exact[:, k0].cpu().numpy()
    e_pred = pred[:, k0].cpu().numpy()
    # screen: recall of the true lowest 10% among the best-ranked 30%
    m = len(e_true)
    target = set(np.argsort(e_true)[: m // 10].tolist())
    chosen = set(np.argsort(e_pred)[: (3 * m) // 10].tolist())
    recall = len(target & chosen) / len(target)
    print(f"screen: recall {recall:.3f} flowing 30% of the queries; |err(n_0)| median "
          f"{np.median(np.abs(e_pred - e_true)):.2e}")
    assert recall >= 0.9
    # gate on the lowest diagonal coefficient: every served answer within
    # 1e-4 (+ the loose flow's own error) of the FP64 flow
    out, ok, tm = sur.screen(th_test, [k0], tol=1e-4)
    ok = ok.cpu().numpy()
    err = (out[:, k0] - exact[:, k0]).abs().cpu().numpy()
    print(f"gate (n_0): served by the network {ok.sum()}/{len(ok)}, timings {tm}")
    assert np.all(err <= 1e-4 + 1e-5)
    if (~ok).any():
        assert np.all(err[~ok] <= 1e-8)
    assert ok.mean() > 0.5
    # the same gate on all 36 diagonal coefficients (reported)
    diag = np.nonzero([int(l) & 0xFFFFFFFF == int(l) >> 32 for l in w.labels])[0]
    e36 = (pred[:, diag] - exact[:, diag]).abs().max(dim=1).values.cpu().numpy()
    print(f"all 36 diagonals: network max error per query median {np.median(e36):.2e}, "
          f"within 1e-4: {np.mean(e36 <= 1e-4):.3f}")

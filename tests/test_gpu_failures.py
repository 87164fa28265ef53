"""Failure detection on the GPU without a GPU fault.

Every failure here is made on purpose in an allowed form: a tensor-core
pipeline wait that nothing will ever satisfy (its copies are withheld by a
host-armed flag) and that gives up after about a second; step-size control
driven below its floor; a step budget that runs out; a device allocation
far larger than any GPU.  Each must come back as its cut_status, and the
same process must keep computing correct results afterwards.
"""
import numpy as np
import pytest

from gpu_util import graph_for, np64
from cut_inputs import workload, batched_parameters

pytestmark = pytest.mark.gpu


def test_pipeline_wait_timeout_is_reported_and_the_context_stays_usable():
    import time
    import paper_2609_14831_b300 as cg
    rng = np.random.default_rng(90)
    m = cg.MLP(32, 128, 64, seed=90, device=0)
    X = rng.normal(size=(256, 32)).astype(np.float32)
    y0 = m.forward(X).cpu().numpy()
    m.status()
    m.inject_stall(True)
    t0 = time.time()
    m.forward(X)
    with pytest.raises(cg.CutError) as e:
        m.status()
    assert e.value.name == "TIMEOUT"
    assert time.time() - t0 < 60
    m.inject_stall(False)
    y1 = m.forward(X).cpu().numpy()
    m.status()                                   # reported once, then clean
    np.testing.assert_array_equal(y1, y0)


def test_step_size_underflow_is_reported():
    import torch
    import paper_2609_14831_b300 as cg
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    with pytest.raises(cg.CutError) as e:
        G.flow(w.h, w.observables, method="dp45", s0=0.0, s1=1.0, ds=1e-2, rtol=1e-300, atol=1e-300)
    assert e.value.name == "STEP_UNDERFLOW"
    H = batched_parameters(w.labels, 8, 5, seed=91)
    X = np.stack([np.stack(w.observables)] * 5)
    _, _, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="dp45",
                                         s0=0.0, s1=1.0, ds=1e-2, rtol=1e-300, atol=1e-300)
    assert np.all(status.cpu().numpy() == 8)     # CUT_ERR_STEP_UNDERFLOW per instance
    # the next flow is unaffected
    hs, _, st, _ = G.flow(w.h, w.observables, method="rk4", s0=0.0, s1=0.01, ds=0.005)
    assert st["steps"] == 2 and np.all(np.isfinite(np64(hs)))


def test_step_limit_is_reported():
    import torch
    import paper_2609_14831_b300 as cg
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    with pytest.raises(cg.CutError) as e:
        G.flow(w.h, w.observables, method="dp45", s0=0.0, s1=10.0, ds=1e-2, rtol=1e-10, atol=w.atol, max_steps=3)
    assert e.value.name == "MAX_STEPS"
    H = batched_parameters(w.labels, 8, 5, seed=92)
    X = np.stack([np.stack(w.observables)] * 5)
    _, _, steps, status = G.flow_batched(torch.tensor(H), torch.tensor(X), precision="fp64", method="dp45",
                                         s0=0.0, s1=10.0, ds=1e-2, rtol=1e-10, atol=w.atol, max_steps=3)
    assert np.all(status.cpu().numpy() == 9)     # CUT_ERR_MAX_STEPS per instance
    assert np.all(steps.cpu().numpy() <= 3)


def test_allocation_failure_is_reported_and_the_context_stays_usable():
    import paper_2609_14831_b300 as cg
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    want_dh, _ = G.rhs(w.h, w.observables)
    want_dh = np64(want_dh)
    n = len(w.h)
    # checkpoint segments of 2^31 - 1 steps: a workspace of tens of terabytes
    with pytest.raises(cg.CutError) as e:
        G.flow_vjp(w.h, w.observables, np.ones(n), [np.ones(n)] * 2, method="rk4", s0=0.0, s1=0.01, ds=1e-3,
                   checkpoint_every=2 ** 31 - 1)
    assert e.value.name == "OUT_OF_MEMORY"
    dh, _ = G.rhs(w.h, w.observables)
    np.testing.assert_array_equal(np64(dh), want_dh)

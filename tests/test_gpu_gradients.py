"""Gradients of flowed coefficients with respect to Hamiltonian parameters
through torch.autograd and the library's checkpointed discrete adjoint.

h0(theta) = h_ref + P theta with 32 parameter directions (8 orbital
energies + 24 unit-norm two-body directions); J = flowed coefficient of n_0
(the lowest orbital) after the DP45 flow of the 8-spin-orbital model to
s = 10, checkpoints every 64 steps.  Checked against central differences
(h = 1e-6) on the same accepted step sequence: relative 1e-6 (difference
truncation ~h^2, rounding ~1e-16/h).
"""
import numpy as np
import pytest

from gpu_util import graph_for, np64
from cut_inputs import make_label, parameter_directions, workload

pytestmark = pytest.mark.gpu


def test_autograd_gradient_matches_central_differences():
    import torch
    from paper_2609_14831_b300 import autograd as ag
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    dev = G.device
    P = torch.tensor(parameter_directions(w.labels, 8), device=dev)
    href = torch.tensor(w.h, device=dev)
    x0 = torch.tensor(np.stack(w.observables), device=dev)
    k0 = int(np.nonzero(w.labels == np.uint64(make_label(1, 1)))[0][0])
    opts = dict(method="dp45", s0=0.0, s1=10.0, ds=1e-2, rtol=1e-10, atol=w.atol)
    theta = torch.zeros(32, dtype=torch.float64, device=dev, requires_grad=True)
    hs, xs = ag.flow(G, href + P @ theta, x0, checkpoint_every=64, **opts)
    J = hs[k0]
    J.backward()
    grad = np64(theta.grad)
    steps = ag._Flow  # noqa: F841  (keep the module referenced)
    # frozen step sequence of the forward flow for the differences
    _, _, st, accepted = G.flow(w.h, list(w.observables), **opts)
    assert st["steps"] > 64            # more than one checkpoint segment
    h = 1e-6
    fd = np.zeros(32)
    Pn = np64(P)
    for c in range(32):
        vals = []
        for sgn in (1, -1):
            hp, _, _, _ = G.flow(w.h + sgn * h * Pn[:, c], list(w.observables), method="dp45", s0=0.0, s1=10.0,
                                 replay=accepted)
            vals.append(np64(hp)[k0])
        fd[c] = (vals[0] - vals[1]) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(grad - fd)) <= 1e-6 * scale, (grad[:4], fd[:4])

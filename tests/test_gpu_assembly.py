"""Multi-operator assembly: combinations of a transformed operator library.

A library of 120 source operators (seeded operands flowed with the
8-spin-orbital model) is transformed once; 1024 seeded combinations with
small integer coefficients are assembled on the GPU and compared with the
oracle's plain sum over the same flowed sources (FP64, relative 1e-14), and
two runs give identical bits.
"""
import numpy as np
import pytest

from gpu_util import assert_close, graph_for, np64
from cut_inputs import workload

pytestmark = pytest.mark.gpu


def test_assembly_of_1024_combinations_from_120_sources():
    import torch
    import paper_2609_14831_b300 as cg
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    rng = np.random.default_rng(90)
    n = len(w.labels)
    src0 = rng.normal(size=(120, n))
    # transform the library once: the batched flow carries up to 3 operands,
    # so flow the sources three at a time alongside the same Hamiltonian
    H = torch.tensor(np.stack([w.h] * 40))
    X = torch.tensor(src0.reshape(40, 3, n))
    _, Xs, _, status = G.flow_batched(H, X, precision="fp64", method="rk4", s0=0.0, s1=0.5, ds=0.01)
    assert int(status.abs().max()) == 0
    lib_t = Xs.reshape(120, n).contiguous()
    C = rng.integers(-3, 4, size=(1024, 120)).astype(np.float64)
    out = cg.assemble(lib_t, torch.tensor(C, device=lib_t.device))
    out2 = cg.assemble(lib_t, torch.tensor(C, device=lib_t.device))
    assert torch.equal(out, out2)
    ref = C @ np64(lib_t)
    assert_close(np64(out).ravel(), ref.ravel(), rtol=1e-13, what="assembly")

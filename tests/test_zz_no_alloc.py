"""cut_rhs_noalloc: the right-hand side for callers that may not allocate.

Some callers cannot ask the CUDA allocator for memory while they run: a
serving or real-time loop that fixed its memory at start-up, or a host
program whose device memory is managed by another component.  cut_rhs
borrows a temporary generator buffer from the stream-ordered allocator;
cut_rhs_noalloc uses a fixed array inside the library instead.  This file
checks, through the C ABI, that two calls in a row give the results of
cut_rhs (within the parity tolerance of the other GPU tests), including a
second graph that reuses the array the first one left behind.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import RTOL, assert_close, graph_for, np64
from cut_inputs import ALG_FERMION, cfg2_registry, dipole_operator, molecular_hamiltonian, number_operator, workload

pytestmark = pytest.mark.gpu


def _noalloc(G, h, xs):
    import torch
    import paper_2609_14831_b300 as cg
    h = torch.as_tensor(h, dtype=torch.float64, device=G.device).contiguous()
    x = torch.stack([torch.as_tensor(v, dtype=torch.float64, device=G.device) for v in xs]).contiguous()
    dh = torch.empty_like(h)
    dx = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    rc = cg.lib().cut_rhs_noalloc(G._h, ctypes.c_void_p(h.data_ptr()), len(xs), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(dh.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
    cg.check(rc)
    torch.cuda.synchronize()
    return np64(dh), [np64(v) for v in dx]


def test_noalloc_rhs_matches_cut_rhs_on_two_calls_in_a_row():
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    labels5 = cfg2_registry(5, keep_shared1=0.3, seed=3)
    h5 = molecular_hamiltonian(labels5, 5, seed=60, scale=0.3)
    x5 = [number_operator(labels5, 5), dipole_operator(labels5, 5, seed=60)]
    G5 = graph_for("mol5_3body", ALG_FERMION, 5, labels5)
    rng = np.random.default_rng(61)
    for graph, h, xs in ((G, w.h, w.observables), (G5, h5, x5), (G, w.h + 0.01 * rng.normal(size=len(w.h)),
                                                                 w.observables)):
        want_dh, want_dx = graph.rhs(h, xs)
        for _ in range(2):
            dh, dx = _noalloc(graph, h, xs)
            assert_close(dh, np64(want_dh), rtol=RTOL, what="dh")
            for a, b in zip(dx, want_dx):
                assert_close(a, np64(b), rtol=RTOL, what="dx")


def test_noalloc_rejects_host_only_handles(tmp_path):
    import paper_2609_14831_b300 as cg
    from cut_inputs import pauli_registry
    p = str(tmp_path / "p.cutg")
    cg.build_graph(0, 2, pauli_registry(2), p)
    H = cg.Graph(p, device=-1)
    assert cg.lib().cut_rhs_noalloc(H._h, None, 0, None, None, None, None) == 1


@pytest.mark.parametrize("n_obs", [3, 4, 7])
def test_packed_and_unpacked_operand_gathers_give_the_same_bits(n_obs):
    """cut_rhs packs the operands of each index into 32-byte blocks (one
    gather per block and record; 4 operands fill one block, 5 fill one and a
    part of a second, 8 fill two);
    cut_rhs_noalloc, which may not allocate the packing scratch, gathers each
    operand separately.  Per operand both sum the same records in the same
    order with the same FMAs: the results are equal bit for bit."""
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    rng = np.random.default_rng(62)
    xs = list(w.observables) + [rng.normal(size=len(w.h)) for _ in range(n_obs - 2)]
    want_dh, want_dx = G.rhs(w.h, xs)
    dh, dx = _noalloc(G, w.h, xs)
    np.testing.assert_array_equal(dh, np64(want_dh))
    for a, b in zip(dx, want_dx):
        np.testing.assert_array_equal(a, np64(b))

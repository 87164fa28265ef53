"""Target-range shards on the GPU (records grouped by output, Sec. 2.2).

One process drives `world` shard handles of the same bundle as threads with
an in-process all-gather (each thread synchronises its stream before it
hands its piece over; no kernel waits on another).  The assembled
right-hand side and a 10-step RK4 flow must equal the whole-graph cut_rhs
and cut_flow bit for bit, because every row is summed by the same kernel in
the same order whichever shard holds it.
"""
import threading

import numpy as np
import pytest

from gpu_util import graph_for, np64
from cut_inputs import ALG_FERMION, cfg2_registry, dipole_operator, molecular_hamiltonian, number_operator, workload

pytestmark = pytest.mark.gpu


class ThreadGroup:
    def __init__(self, world):
        self.world = world
        self.slots = [None] * world
        self.bar = threading.Barrier(world)

    def gather_fn(self, rank):
        import torch

        def gather(t):
            torch.cuda.current_stream().synchronize()
            self.slots[rank] = t
            self.bar.wait()
            out = torch.cat(self.slots)
            torch.cuda.current_stream().synchronize()
            self.bar.wait()
            return out
        return gather


def _sharded(path, world, h, xs, s1, ds, arith="fp64"):
    import torch
    from paper_2609_14831_b300.sharded import DeviceShard, ShardedRHS
    grp = ThreadGroup(world)
    out, err = [None] * world, []

    def run(r):
        try:
            ex = DeviceShard(path, 0, r, world)
            ex.set_arithmetic(arith)
            sh = ShardedRHS(ex, grp.gather_fn(r))
            Y = torch.tensor(np.stack([h] + list(xs)), device="cuda")
            DY = torch.empty_like(Y)
            sh.rhs(Y, DY)
            dy = np64(DY)
            sh.flow_rk4(Y, 0.0, s1, ds)
            out[r] = (dy, np64(Y), ex.R_local, ex.device_bytes)
            ex.close()
        except Exception as e:          # surface thread failures in the test
            err.append(e)
            grp.bar.abort()
    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(600)
    assert not err, err
    return out


@pytest.mark.parametrize("case,world", [("mol8", 2), ("mol8", 3), ("mol5_3body", 2), ("pauli6", 3)])
def test_shards_reproduce_whole_graph_rhs_and_flow(case, world):
    """pauli6: 4,096 long rows, which the commutator stage cuts into pieces;
    every shard cuts its rows as the whole graph does."""
    if case == "mol8":
        w = workload("molecular_8so")
        alg, nm, labels, h, xs = w.alg, w.nmodes, w.labels, w.h, list(w.observables)
    elif case == "pauli6":
        from cut_inputs import ALG_PAULI, pauli_registry
        labels = pauli_registry(6)
        alg, nm = ALG_PAULI, 6
        rng = np.random.default_rng(78)
        h = rng.normal(size=len(labels)) * 0.1
        xs = [rng.normal(size=len(labels))]
    else:
        labels = cfg2_registry(5, keep_shared1=0.3, seed=3)
        alg, nm = ALG_FERMION, 5
        h = molecular_hamiltonian(labels, 5, seed=60, scale=0.3)
        xs = [number_operator(labels, 5), dipole_operator(labels, 5, seed=60)]
    G = graph_for(case, alg, nm, labels)
    path = G.path
    dh, dx = G.rhs(h, xs)
    want_rhs = np.stack([np64(dh)] + [np64(v) for v in dx])
    hs, xo, st, _ = G.flow(h, xs, method="rk4", s0=0.0, s1=0.05, ds=0.005)
    want_y = np.stack([np64(hs)] + [np64(v) for v in xo])
    out = _sharded(path, world, h, xs, 0.05, 0.005)
    R = G.R_g + G.R_L
    for r, (dy, y, R_local, _) in enumerate(out):
        np.testing.assert_array_equal(dy, want_rhs, err_msg=f"rank {r} rhs")
        np.testing.assert_array_equal(y, want_y, err_msg=f"rank {r} flow")
        assert R_local < R
    assert sum(o[2] for o in out) == R          # every record on exactly one shard


def test_shard_handles_refuse_whole_graph_calls():
    import ctypes
    import torch
    import paper_2609_14831_b300 as cg
    from paper_2609_14831_b300.sharded import DeviceShard
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    ex = DeviceShard(G.path, 0, 1, 2)
    h = torch.tensor(w.h, device="cuda")
    dh = torch.empty_like(h)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    assert cg.lib().cut_rhs(ex._h, P(h), 0, None, P(dh), None, None, None) == 1
    assert cg.lib().cut_rhs_noalloc(ex._h, P(h), 0, None, P(dh), None, None) == 1
    ex.close()


def test_double_float_shards_reproduce_the_whole_graph():
    """The double-float commutator stage on 2 shards equals the whole
    graph's double-float right-hand side and RK4 flow bit for bit."""
    w = workload("molecular_8so")
    G = graph_for("mol8", w.alg, w.nmodes, w.labels)
    G.set_arithmetic("df64")
    try:
        dh, dx = G.rhs(w.h, list(w.observables))
        want_rhs = np.stack([np64(dh)] + [np64(v) for v in dx])
        hs, xo, st, _ = G.flow(w.h, list(w.observables), method="rk4", s0=0.0, s1=0.05, ds=0.005)
        want_y = np.stack([np64(hs)] + [np64(v) for v in xo])
    finally:
        G.set_arithmetic("fp64")
    out = _sharded(G.path, 2, w.h, list(w.observables), 0.05, 0.005, arith="df64")
    for r, (dy, y, _, _) in enumerate(out):
        np.testing.assert_array_equal(dy, want_rhs, err_msg=f"rank {r} rhs")
        np.testing.assert_array_equal(y, want_y, err_msg=f"rank {r} flow")

"""Host logic of the benchmark's multi-rank path on CPU (gloo, world 2)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    out[rank] = ms
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 15.0


def test_job_throughput_is_weak_scaling_sum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(1000, 2.0, 1) == 500000.0
    assert bench.job_throughput(1000, 2.0, 4) == 2000000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_sample_record_counts_match_fresh_builds(tmp_path):
    """The record counts the CPU baseline divides by are those of the graphs
    cut_build compiles for the two sample workloads."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_2609_14831_b300 as cg
    from cut_inputs import workload
    for name, seed in (("stress_7so", 2), ("molecular_8so", 1)):
        w = workload(name, seed=seed)
        st = cg.build_graph(w.alg, w.nmodes, w.labels, str(tmp_path / f"{name}.cutg"))
        assert st["R_g"] + st["R_L"] == bench.SAMPLE_RECORDS[name], name


def test_parallel_oracle_rhs_equals_the_oracle():
    """The process-pool split of the oracle's right-hand side (by the labels
    of each operand; the commutator is linear in X) gives the oracle's RHS."""
    import multiprocessing as mp
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from cut_inputs import workload
    w = workload("molecular_4so")
    with mp.get_context("spawn").Pool(2) as pool:
        got = bench.oracle_rhs_parallel(pool, 3, w.alg, w.nmodes, w.labels, w.h, w.observables)
    dh, dxs = oracle.rhs(w.alg, w.nmodes, w.labels, w.h, w.observables)
    for g, want in zip(got, [dh] + list(dxs)):
        np.testing.assert_allclose(g, want, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(want))))


def test_launch_count_follows_the_stage_structure():
    """The bench's gpu_launches claim for the timed RK4 flow: on the stress
    graph (3.5e6 generator records, three operands) a step is four stages of
    generator+packing and commutator launches, three stage inputs and the
    final combination; an ncu launch list of the timed region counts
    40 + 40 + 40 + 1 for ten steps."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rk4_launches(10, 3, 3456464) == 121
    # a small graph: stage input, packing and generator fused into one launch
    assert bench.rk4_launches(10, 3, 4648) == 10 * (4 * 2 + 1) + 1
    # nine operands: generator, then two commutator passes of up to eight
    assert bench.rk4_launches(1, 9, 3456464) == 4 * (1 + 2) + 3 + 1 + 1

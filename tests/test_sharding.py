"""Target-range sharding (records grouped by output, paper Sec. 2.2) on CPU.

The partition of each stage into record-balanced contiguous row ranges is
the library's (cut_graph_partition, host-only handle); the orchestration is
the package's ShardedRHS, run by two gloo ranks.  Each rank applies only the
records of its own rows with a plain numpy executor (test infrastructure:
the library itself has no CPU traversal), all-gathers xi and the right-hand
side, and advances RK4.  Both ranks must reproduce the single-rank right-hand
side and a 10-step RK4 flow bit for bit, and the flow must match the oracle.
"""
import os
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class NumpyShard:
    """Applies the records of one rank's rows in numpy (fixed order per row)."""

    def __init__(self, path, rank, world):
        import ctypes
        import paper_2609_14831_b300 as cg
        from paper_2609_14831_b300.sharded import partition
        G = cg.Graph(path, device=-1)
        self.n, self.n_g, self.rank, self.world = G.n, G.n_g, rank, world
        self.gen_bounds = partition(G._h, 0, world)
        self.comm_bounds = partition(G._h, 1, world)
        num, den = G.weights()
        w = num.astype(np.float64) / den
        self.st = []
        for stage, b in ((0, self.gen_bounds), (1, self.comm_bounds)):
            rp, a, bb, code = G.records(stage)
            lo, hi = int(b[rank]), int(b[rank + 1])
            self.st.append((rp[lo:hi + 1] - rp[lo], a[rp[lo]:rp[hi]].astype(np.int64),
                            bb[rp[lo]:rp[hi]].astype(np.int64), w[code[rp[lo]:rp[hi]]]))
        G.close()

    def empty(self, *shape):
        return torch.empty(*shape, dtype=torch.float64)

    def generator(self, h, out):
        rp, i, j, w = self.st[0]
        h = h.numpy()
        t = w * h[i] * h[j]
        o = out.numpy()
        for r in range(len(rp) - 1):
            o[r] = np.sum(t[rp[r]:rp[r + 1]])

    def commutator(self, xi, X, out):
        rp, a, j, w = self.st[1]
        xi, X = xi.numpy(), X.numpy()
        rows = len(rp) - 1
        o = out.numpy().reshape(X.shape[0], -1)
        c = w * xi[a]
        for q in range(X.shape[0]):
            t = c * X[q][j]
            for r in range(rows):
                o[q, r] = np.sum(t[rp[r]:rp[r + 1]])

    def combine(self, base, Ks, cs, ds, out):
        v = base.numpy().copy()
        for K, c in zip(Ks, cs):
            if c != 0.0:
                v += (c * ds) * K.numpy()
        out.numpy()[...] = v


def _problem():
    from cut_inputs import ALG_FERMION, cfg2_registry, dipole_operator, molecular_hamiltonian, number_operator
    labels = cfg2_registry(4, keep_shared1=1.0, seed=7)
    h = molecular_hamiltonian(labels, 4, seed=70, scale=0.3)
    xs = [number_operator(labels, 4), dipole_operator(labels, 4, seed=70)]
    return ALG_FERMION, 4, labels, h, xs


def _run(path, rank, world, gather):
    from paper_2609_14831_b300.sharded import ShardedRHS
    alg, nm, labels, h, xs = _problem()
    ex = NumpyShard(path, rank, world)
    sh = ShardedRHS(ex, gather)
    Y = torch.tensor(np.stack([h] + xs))
    DY = torch.empty_like(Y)
    sh.rhs(Y, DY)
    sh.flow_rk4(Y, 0.0, 0.05, 0.005)
    return DY.numpy().copy(), Y.numpy().copy(), ex


def _worker(rank, world, port, path, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2609_14831_b300.sharded import torch_all_gather
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dy, y, _ = _run(path, rank, world, torch_all_gather())
    np.save(os.path.join(outdir, f"dy{rank}.npy"), dy)
    np.save(os.path.join(outdir, f"y{rank}.npy"), y)
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def bundle(tmp_path_factory):
    import paper_2609_14831_b300 as cg
    alg, nm, labels, h, xs = _problem()
    p = str(tmp_path_factory.mktemp("shard") / "g.cutg")
    cg.build_graph(alg, nm, labels, p)
    return p


def test_partition_is_contiguous_and_record_balanced(bundle):
    import paper_2609_14831_b300 as cg
    from paper_2609_14831_b300.sharded import partition
    G = cg.Graph(bundle, device=-1)
    for stage in (0, 1):
        rp = G.records(stage)[0]
        rows, R = len(rp) - 1, int(rp[-1])
        longest = int(np.max(np.diff(rp)))
        for parts in (1, 2, 3, 7, rows + 5):
            b = partition(G._h, stage, parts)
            assert b[0] == 0 and b[-1] == rows and np.all(np.diff(b) >= 0)
            got = rp[b[1:]] - rp[b[:-1]]
            assert got.sum() == R
            # every part within one row of its share
            assert np.all(np.abs(got - R / parts) <= longest + 1), (stage, parts)
    G.close()


def test_two_gloo_ranks_reproduce_the_single_rank_rhs_and_rk4_flow(bundle, tmp_path):
    import oracle
    dy1, y1, ex = _run(bundle, 0, 1, lambda t: t.clone())
    # both ranks hold records of both stages: the split is real
    for r in range(2):
        part = NumpyShard(bundle, r, 2)
        assert len(part.st[0][1]) > 0 and len(part.st[1][1]) > 0
        assert 0 < part.comm_bounds[1] < part.comm_bounds[2]
    ctx = mp.get_context("spawn")
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, bundle, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"dy{r}.npy"), dy1)
        np.testing.assert_array_equal(np.load(tmp_path / f"y{r}.npy"), y1)
    # and the single-rank path is the method: the oracle's RHS and RK4 flow
    alg, nm, labels, h, xs = _problem()
    n = len(labels)
    want_dh, want_dx = oracle.rhs(alg, nm, labels, h, xs)
    for got, want in zip(dy1, [want_dh] + list(want_dx)):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(want))))
    f = oracle.stacked_rhs(alg, nm, labels, 2)
    y = oracle.rk4_flow(f, np.concatenate([h] + xs), 0.005, 10)
    np.testing.assert_allclose(y1.ravel(), y, rtol=0, atol=1e-12 * np.max(np.abs(y)))


def _worker_fail(rank, world, port, path, outdir):
    """Rank 1 leaves before its first exchange; rank 0 must get an error from
    the all-gather within the group's timeout instead of hanging."""
    import datetime
    import time as _time
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2609_14831_b300.sharded import ShardedRHS, torch_all_gather
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        open(os.path.join(outdir, "left1"), "w").close()
        os._exit(0)                              # leaves between steps, nothing in flight
    alg, nm, labels, h, xs = _problem()
    sh = ShardedRHS(NumpyShard(path, rank, world), torch_all_gather())
    Y = torch.tensor(np.stack([h] + xs))
    t0 = _time.time()
    try:
        sh.rhs(Y, torch.empty_like(Y))
        res = "no error"
    except Exception as e:                       # the exchange fails on the host
        res = f"error after {_time.time() - t0:.1f} s: {type(e).__name__}"
    open(os.path.join(outdir, "rank0.txt"), "w").write(res)
    os._exit(0)


def test_a_rank_that_leaves_is_detected_by_the_others(bundle, tmp_path):
    ctx = mp.get_context("spawn")
    port = 29700 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, bundle, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = (tmp_path / "rank0.txt").read_text()
    print(res)
    assert res.startswith("error after")
    assert float(res.split()[2]) < 60


def test_three_gloo_ranks_with_uneven_pieces_reproduce_the_single_rank_flow(bundle, tmp_path):
    """Three ranks: the record-balanced row ranges have different lengths, so
    the all-gather pads them to the longest and each rank must cut its
    neighbours' pieces back out in rank order.  Same bits as one rank."""
    dy1, y1, _ = _run(bundle, 0, 1, lambda t: t.clone())
    lens = [np.diff(NumpyShard(bundle, 0, 3).comm_bounds)]
    assert len(set(lens[0].tolist())) > 1                 # the pieces differ in length
    ctx = mp.get_context("spawn")
    port = 29700 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 3, port, bundle, str(tmp_path))) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(3):
        np.testing.assert_array_equal(np.load(tmp_path / f"dy{r}.npy"), dy1)
        np.testing.assert_array_equal(np.load(tmp_path / f"y{r}.npy"), y1)

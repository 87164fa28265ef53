"""Target-range sharding of one operation graph over a process group.

Records are grouped by output (paper Sec. 2.2), so each stage's outputs split
into contiguous, record-balanced row ranges (``cut_graph_partition``).  A rank
holds one range of the generator stage and one of the commutator stage
(``cut_graph_load_shard``: about 1/world of the records on its device) and
every right-hand side runs as

    xi piece   = generator stage of the rank's rows        (cut_shard_generator)
    xi         = all-gather of the pieces                   (collective)
    F piece    = commutator stage of the rank's rows        (cut_shard_commutator)
    F          = all-gather of the pieces                   (collective)

after which every rank holds the whole right-hand side and advances the same
Runge-Kutta state (``cut_combine``, the kernel ``cut_flow`` uses).  Each row
is summed exactly as the whole graph sums it, so the flow equals the
single-device ``cut_flow`` bit for bit.

This module only moves data: the stages and the RK combinations run in
libcut.so; the all-gather is the process group's (NCCL between GPUs, gloo on
host tensors).  The orchestration (`ShardedRHS`) takes any executor with the
same three calls, which is how the host-side logic is tested on CPU ranks.
"""
import ctypes

import numpy as np

from . import GraphDesc, VP, _ptr, _stream, _torch, check, lib

# classical RK4 (the tableau cut_flow uses)
RK4_A = [[], [0.5], [0.0, 0.5], [0.0, 0.0, 1.0]]
RK4_B = [1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6]


def partition(graph_handle, stage, parts):
    """Record-balanced row bounds [parts + 1] of a stage (whole-graph handle)."""
    b = np.empty(parts + 1, dtype=np.int64)
    check(lib().cut_graph_partition(graph_handle, int(stage), int(parts), b.ctypes.data))
    return b


class DeviceShard:
    """One rank's shard of a graph on a CUDA device (the libcut.so executor).

    Attributes: n, n_g, gen_bounds / comm_bounds (row bounds of every rank),
    rank, world."""

    def __init__(self, path, device, rank, world):
        import os
        L = lib()
        self._h = VP()
        check(L.cut_graph_load_shard(os.fsencode(path), int(device), int(rank), int(world), 0,
                                     ctypes.byref(self._h)))
        d = GraphDesc()
        check(L.cut_graph_query(self._h, ctypes.byref(d)))
        self.n, self.n_g = d.n, d.n_g
        self.rank, self.world = d.shard_rank, d.shard_world
        self.device_index = int(device)
        # the bounds of every rank, from a host-only handle of the same bundle
        whole = VP()
        check(L.cut_graph_load(os.fsencode(path), -1, 0, ctypes.byref(whole)))
        try:
            self.gen_bounds = partition(whole, 0, world)
            self.comm_bounds = partition(whole, 1, world)
        finally:
            L.cut_graph_free(whole)
        assert (self.gen_bounds[rank], self.gen_bounds[rank + 1]) == (d.gen_lo, d.gen_hi)
        assert (self.comm_bounds[rank], self.comm_bounds[rank + 1]) == (d.comm_lo, d.comm_hi)
        self.R_local = d.R_g + d.R_L
        self.device_bytes = d.device_bytes

    @property
    def device(self):
        return _torch().device("cuda", self.device_index)

    def close(self):
        if self._h:
            lib().cut_graph_free(self._h)
            self._h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, *shape):
        torch = _torch()
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    def set_arithmetic(self, mode):
        """'fp64' or 'df64' for this shard's commutator stage (as Graph)."""
        check(lib().cut_graph_set_arithmetic(self._h, {"fp64": 0, "df64": 1}[mode]))

    def generator(self, h, out, stream=None):
        """out[gen_hi - gen_lo] = xi of this shard's generator rows."""
        check(lib().cut_shard_generator(self._h, _ptr(h), _ptr(out), _stream(stream)))

    def commutator(self, xi, X, out, stream=None):
        """out[nops][comm_hi - comm_lo] = L(h) X_o on this shard's rows."""
        check(lib().cut_shard_commutator(self._h, _ptr(xi), X.shape[0], _ptr(X), _ptr(out), _stream(stream)))

    def combine(self, base, Ks, cs, ds, out, stream=None):
        """out = base + sum_s (c_s ds) K_s (the RK combination of cut_flow)."""
        nk = len(Ks)
        K = (ctypes.c_void_p * max(1, nk))(*[k.data_ptr() for k in Ks])
        c = (ctypes.c_double * max(1, nk))(*cs)
        check(lib().cut_combine(base.numel(), _ptr(base), nk, K, c, float(ds), _ptr(out), _stream(stream)))


def torch_all_gather(group=None):
    """All-gather of equal-length 1-D tensors through torch.distributed
    (one all_gather_into_tensor on NCCL; a list all_gather on gloo)."""
    import torch.distributed as dist
    torch = _torch()
    nccl = dist.get_backend(group) == "nccl"
    world = dist.get_world_size(group)

    def gather(t):
        t = t.contiguous()
        out = torch.empty(world * t.numel(), dtype=t.dtype, device=t.device)
        if nccl:
            dist.all_gather_into_tensor(out, t, group=group)
        else:
            dist.all_gather(list(out.view(world, -1).unbind(0)), t, group=group)
        return out
    return gather


class ShardedRHS:
    """Right-hand sides and RK4 flows of one shard group.

    ex: an executor (DeviceShard, or any object with n, n_g, rank, world,
    gen_bounds, comm_bounds, empty(), generator(), commutator(), combine());
    all_gather: maps this rank's 1-D tensor of length m to the world's
    [world * m] concatenation (rank order)."""

    def __init__(self, ex, all_gather):
        self.ex = ex
        self.gather = all_gather
        gb, cb = np.asarray(ex.gen_bounds), np.asarray(ex.comm_bounds)
        self.gen_len = np.diff(gb)
        self.comm_len = np.diff(cb)
        self.gen_pad = max(1, int(self.gen_len.max()))
        self.comm_pad = max(1, int(self.comm_len.max()))
        self.gb, self.cb = gb, cb

    def _gather_pieces(self, piece, lens, bounds, pad, width, out):
        """Pieces of `width` rows-major vectors ([width][len_r] on rank r) into
        out[width][total] (every rank gets the same bits)."""
        r = self.ex.rank
        buf = self.ex.empty(width * pad)
        buf.zero_()
        if lens[r]:
            buf.view(width, pad)[:, :lens[r]].copy_(piece.view(width, lens[r]))
        allp = self.gather(buf).view(len(lens), width, pad)
        for q in range(len(lens)):
            if lens[q]:
                out[:, bounds[q]:bounds[q + 1]].copy_(allp[q, :, :lens[q]])
        return out

    def rhs(self, Y, DY, xi=None):
        """DY[nops][n] = F(Y) for the stacked state Y[nops][n] (Y[0] = h)."""
        ex, r = self.ex, self.ex.rank
        nops = Y.shape[0]
        xi_part = ex.empty(max(1, int(self.gen_len[r])))
        ex.generator(Y[0], xi_part)
        xi = ex.empty(1, max(1, ex.n_g)) if xi is None else xi.view(1, -1)
        self._gather_pieces(xi_part, self.gen_len, self.gb, self.gen_pad, 1, xi)
        part = ex.empty(nops * max(1, int(self.comm_len[r])))
        ex.commutator(xi.view(-1), Y, part)
        self._gather_pieces(part, self.comm_len, self.cb, self.comm_pad, nops, DY)
        return DY

    def flow_rk4(self, Y, s0, s1, ds):
        """Fixed-step RK4 of the stacked state in place; the step count and
        size follow cut_flow (N = round((s1 - s0) / ds), ds = (s1 - s0) / N)."""
        N = int(np.floor((s1 - s0) / ds + 0.5))     # llround, as cut_flow
        if N < 1:
            N = 1 if s1 > s0 else 0
        if N == 0:
            return Y, 0
        dse = (s1 - s0) / N
        ex = self.ex
        K = [ex.empty(*Y.shape) for _ in range(4)]
        U = ex.empty(*Y.shape)
        for _ in range(N):
            for i in range(4):
                if i == 0:
                    self.rhs(Y, K[0])
                    continue
                ex.combine(Y, [K[j] for j in range(i)], RK4_A[i], dse, U)
                self.rhs(U, K[i])
            ex.combine(Y, K, RK4_B, dse, Y)
        return Y, N

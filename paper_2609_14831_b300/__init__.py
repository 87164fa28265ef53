"""B300-native engine for compile-once CUT operation graphs (Python binding).

This module only marshals arguments: every step of the graph build, the
right-hand side, the adjoint and the flows runs inside libcut.so (C++ and
sm_103a CUDA kernels behind the C ABI of include/cut.h).  PyTorch provides
device memory and streams.  If libcut.so is missing the import of the
library fails loudly; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcut.so")

ALG_PAULI, ALG_FERMION = 0, 1
RK4, DP45 = 0, 1
FP64, FP32REC_FP64STATE = 0, 1

STATUS_NAMES = ["OK", "INVALID_ARG", "IO", "FORMAT", "CHECKSUM", "OUT_OF_MEMORY", "CUDA",
                "NONFINITE", "STEP_UNDERFLOW", "MAX_STEPS", "TIMEOUT", "UNSUPPORTED"]


class CutError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"CUT_ERR_{name}: {msg}")
        self.status = status
        self.name = name


class BuildOpts(ctypes.Structure):
    _fields_ = [("algebra", ctypes.c_int), ("nmodes", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("threads", ctypes.c_int), ("diagnostics", ctypes.c_int)]


class BuildStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_g", ctypes.c_int64), ("R_g", ctypes.c_int64),
                ("R_L", ctypes.c_int64), ("n_codes", ctypes.c_int),
                ("seconds_count", ctypes.c_double), ("seconds_write", ctypes.c_double),
                ("seconds_total", ctypes.c_double), ("bytes_stored", ctypes.c_int64),
                ("peak_rss_bytes", ctypes.c_int64)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("algebra", ctypes.c_int), ("nmodes", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("n_codes", ctypes.c_int), ("n", ctypes.c_int64), ("n_g", ctypes.c_int64),
                ("R_g", ctypes.c_int64), ("R_L", ctypes.c_int64), ("sha256", ctypes.c_uint8 * 32),
                ("device_bytes", ctypes.c_int64), ("record_bytes", ctypes.c_int64),
                ("n_out", ctypes.c_int64), ("R_C", ctypes.c_int64),
                ("shard_rank", ctypes.c_int), ("shard_world", ctypes.c_int),
                ("gen_lo", ctypes.c_int64), ("gen_hi", ctypes.c_int64),
                ("comm_lo", ctypes.c_int64), ("comm_hi", ctypes.c_int64)]


class FlowOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("s0", ctypes.c_double), ("s1", ctypes.c_double),
                ("ds", ctypes.c_double), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("replay_steps", ctypes.POINTER(ctypes.c_double)),
                ("n_replay", ctypes.c_int64), ("record_steps", ctypes.POINTER(ctypes.c_double)),
                ("record_cap", ctypes.c_int64), ("batch_record_steps", ctypes.c_void_p),
                ("pause_after", ctypes.c_int64)]


class FlowStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rejects", ctypes.c_int64), ("rhs_calls", ctypes.c_int64),
                ("s_final", ctypes.c_double), ("ds_next", ctypes.c_double), ("finished", ctypes.c_int)]


_lib = None
VP = ctypes.c_void_p


def lib():
    """Load libcut.so (built in-tree by build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcut.so is not built ({LIB_PATH}); run paper_2609_14831_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i, i64, st = ctypes.c_int, ctypes.c_int64, ctypes.c_int
    sig = {
        "cut_last_error": (ctypes.c_char_p, []),
        "cut_version": (ctypes.c_char_p, []),
        "cut_build": (st, [ctypes.POINTER(BuildOpts), i64, VP, ctypes.c_char_p, ctypes.POINTER(BuildStats)]),
        "cut_graph_load": (st, [ctypes.c_char_p, i, ctypes.c_uint, ctypes.POINTER(VP)]),
        "cut_graph_free": (st, [VP]),
        "cut_graph_query": (st, [VP, ctypes.POINTER(GraphDesc)]),
        "cut_graph_labels": (st, [VP, VP, VP, VP]),
        "cut_graph_weights": (st, [VP, VP, VP]),
        "cut_graph_outside_labels": (st, [VP, VP]),
        "cut_rhs_outside": (st, [VP, VP, i, VP, VP, VP]),
        "cut_graph_records": (st, [VP, i, VP, VP, VP, VP]),
        "cut_rhs": (st, [VP, VP, i, VP, VP, VP, VP, VP]),
        "cut_rhs_adjoint": (st, [VP, VP, i, VP, VP, VP, VP, VP, VP]),
        "cut_rhs_noalloc": (st, [VP, VP, i, VP, VP, VP, VP]),
        "cut_graph_set_arithmetic": (st, [VP, i]),
        "cut_apply_L": (st, [VP, VP, i, VP, VP, VP]),
        "cut_rhs_jvp": (st, [VP, VP, i, VP, VP, VP, VP, VP, VP]),
        "cut_assemble": (st, [i, i64, VP, i, VP, VP, VP]),
        "cut_flow": (st, [VP, VP, i, VP, ctypes.POINTER(FlowOpts), ctypes.POINTER(FlowStats), VP]),
        "cut_flow_vjp": (st, [VP, VP, i, VP, ctypes.POINTER(FlowOpts), i, VP, VP, VP, VP, VP]),
        "cut_flow_batched": (st, [VP, i, VP, i, VP, i, ctypes.POINTER(FlowOpts), i, VP, VP, VP]),
        "cut_graph_partition": (st, [VP, i, i, VP]),
        "cut_graph_load_shard": (st, [ctypes.c_char_p, i, i, i, ctypes.c_uint, ctypes.POINTER(VP)]),
        "cut_shard_generator": (st, [VP, VP, VP, VP]),
        "cut_shard_commutator": (st, [VP, VP, i, VP, VP, VP]),
        "cut_combine": (st, [i64, VP, i, VP, VP, ctypes.c_double, VP, VP]),
        "cut_measure_fma_rate": (st, [i, i, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "cut_flow_batched_last_tile": (i, []),
        "cut_mlp_create": (st, [i, i, i, ctypes.c_uint64, i, ctypes.POINTER(VP)]),
        "cut_mlp_free": (st, [VP]),
        "cut_mlp_set_output_affine": (st, [VP, VP, VP]),
        "cut_mlp_get_output_affine": (st, [VP, VP, VP]),
        "cut_mlp_set_linear": (st, [VP, VP]),
        "cut_mlp_param_count": (i64, [VP]),
        "cut_mlp_get_params": (st, [VP, VP, i]),
        "cut_mlp_set_params": (st, [VP, VP]),
        "cut_mlp_forward": (st, [VP, i, VP, VP, VP]),
        "cut_mlp_backward": (st, [VP, i, VP, VP, VP, VP]),
        "cut_mlp_adamw_step": (st, [VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, VP]),
        "cut_mlp_status": (st, [VP]),
        "cut_mlp_inject_stall": (st, [VP, i]),
        "cut_mlp_fit_linear": (st, [VP, i, VP, VP, VP, VP]),
        "cut_mlp_ensemble_stats": (st, [i, i, i, VP, VP, VP, VP, VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status):
    if status != 0:
        raise CutError(status, lib().cut_last_error().decode())


def measure_fma_rate(device=0, fp64=True, seconds=0.5):
    """Measured FMA throughput of a device in TFLOP/s (FP64 or FP32)."""
    out = ctypes.c_double(0.0)
    check(lib().cut_measure_fma_rate(int(device), 1 if fp64 else 0, float(seconds), ctypes.byref(out)))
    return out.value


def build_graph(algebra, nmodes, labels, path, max_rank=0, threads=0, diagnostics=False):
    """Compile the operation graph of a registry into a bundle file."""
    labels = np.ascontiguousarray(labels, dtype=np.uint64)
    opts = BuildOpts(int(algebra), int(nmodes), int(max_rank), int(threads), 1 if diagnostics else 0)
    st = BuildStats()
    check(lib().cut_build(ctypes.byref(opts), len(labels), labels.ctypes.data, os.fsencode(path),
                          ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in BuildStats._fields_}


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t, n, name, device):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.float64))
    t = t.to(device=device, dtype=torch.float64).contiguous()
    if t.shape[-1] != n:
        raise ValueError(f"{name}: last dimension {t.shape[-1]} != registry size {n}")
    return t


def assemble(X, C, stream=None):
    """out[m] = sum_i C[m, i] X[i] (multi-operator assembly, FP64, fixed order)."""
    torch = _torch()
    X = X.to(dtype=torch.float64).contiguous()
    C = C.to(device=X.device, dtype=torch.float64).contiguous()
    out = torch.empty(C.shape[0], X.shape[1], dtype=torch.float64, device=X.device)
    check(lib().cut_assemble(X.shape[0], X.shape[1], _ptr(X), C.shape[0], _ptr(C), _ptr(out), _stream(stream)))
    return out


class Graph:
    """A loaded operation graph resident on one CUDA device."""

    def __init__(self, path, device=0, adjoint=False):
        """adjoint=True builds the transposed record orders of the reverse
        traversal at load time (CUT_LOAD_ADJOINT) instead of at the first
        adjoint call."""
        self._h = VP()
        check(lib().cut_graph_load(os.fsencode(path), int(device), 1 if adjoint else 0, ctypes.byref(self._h)))
        self.path = path
        self.device_index = int(device)
        d = GraphDesc()
        check(lib().cut_graph_query(self._h, ctypes.byref(d)))
        self.desc = {f: (bytes(getattr(d, f)).hex() if f == "sha256" else getattr(d, f))
                     for f, _ in GraphDesc._fields_}
        self.n, self.n_g = d.n, d.n_g
        self.R_g, self.R_L = d.R_g, d.R_L
        self.n_out, self.R_C = d.n_out, d.R_C

    def close(self):
        if self._h:
            lib().cut_graph_free(self._h)
            self._h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device(self):
        return _torch().device("cuda", self.device_index)

    # ---- host-side views of the bundle
    def labels(self):
        lab = np.empty(self.n, dtype=np.uint64)
        gl = np.empty(max(1, self.n_g), dtype=np.uint64)
        dg = np.empty(self.n, dtype=np.uint8)
        check(lib().cut_graph_labels(self._h, lab.ctypes.data, gl.ctypes.data, dg.ctypes.data))
        return lab, gl[:self.n_g], dg.astype(bool)

    def weights(self):
        nc = self.desc["n_codes"]
        num = np.empty(nc, dtype=np.int32)
        den = np.empty(nc, dtype=np.int32)
        check(lib().cut_graph_weights(self._h, num.ctypes.data, den.ctypes.data))
        return num, den

    def outside_labels(self):
        out = np.empty(max(1, self.n_out), dtype=np.uint64)
        check(lib().cut_graph_outside_labels(self._h, out.ctypes.data))
        return out[:self.n_out]

    def rhs_outside(self, h, xs=(), stream=None):
        """Outside-space diagnostic C_q for H and the operands: [1 + n_obs, n_out]."""
        torch = _torch()
        h = _dev_f64(h, self.n, "h", self.device)
        n_obs = len(xs)
        x = torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]) if n_obs else None
        c = torch.empty(1 + n_obs, max(1, self.n_out), dtype=torch.float64, device=self.device)
        check(lib().cut_rhs_outside(self._h, _ptr(h), n_obs, _ptr(x), _ptr(c), _stream(stream)))
        return c[:, :self.n_out]

    def records(self, stage):
        rows = (self.n_g, self.n, self.n_out)[stage]
        R = (self.R_g, self.R_L, self.R_C)[stage]
        rp = np.empty(rows + 1, dtype=np.int64)
        a = np.empty(max(R, 1), dtype=np.int32)
        b = np.empty(max(R, 1), dtype=np.int32)
        c = np.empty(max(R, 1), dtype=np.uint8)
        check(lib().cut_graph_records(self._h, int(stage), rp.ctypes.data, a.ctypes.data,
                                      b.ctypes.data, c.ctypes.data))
        return rp, a[:R], b[:R], c[:R]

    # ---- device traversals
    def rhs(self, h, xs=None, want_xi=False, stream=None):
        """(dh, dxs[, xi]) = P[eta(h), H], P[eta(h), X_o]; tensors on this device."""
        torch = _torch()
        h = _dev_f64(h, self.n, "h", self.device)
        n_obs = 0 if xs is None else len(xs)
        x = _dev_f64(torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]), self.n, "x",
                     self.device) if n_obs else None
        dh = torch.empty_like(h)
        dx = torch.empty_like(x) if n_obs else None
        xi = torch.empty(max(1, self.n_g), dtype=torch.float64, device=self.device) if want_xi else None
        check(lib().cut_rhs(self._h, _ptr(h), n_obs, _ptr(x), _ptr(dh), _ptr(dx), _ptr(xi),
                            _stream(stream)))
        out = (dh, list(dx) if n_obs else [])
        return out + (xi[:self.n_g],) if want_xi else out

    def set_arithmetic(self, mode):
        """'fp64' (default) or 'df64' (FP32-pair products and sums)."""
        check(lib().cut_graph_set_arithmetic(self._h, {"fp64": 0, "df64": 1}[mode]))

    def apply_L(self, xi, xs, stream=None):
        """L(h) x_o for generator coordinates xi (commutator stage alone)."""
        torch = _torch()
        xi = xi.to(device=self.device, dtype=torch.float64).contiguous()
        x = torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]).contiguous()
        dx = torch.empty_like(x)
        check(lib().cut_apply_L(self._h, _ptr(xi), x.shape[0], _ptr(x), _ptr(dx), _stream(stream)))
        return list(dx)

    def rhs_jvp(self, h, xs, dh, dxs, stream=None):
        """Directional derivative of rhs() along (dh, dxs)."""
        torch = _torch()
        h = _dev_f64(h, self.n, "h", self.device)
        dh = _dev_f64(dh, self.n, "dh", self.device)
        n_obs = len(xs)
        x = torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]) if n_obs else None
        dx = torch.stack([_dev_f64(v, self.n, "dx", self.device) for v in dxs]) if n_obs else None
        oh = torch.empty_like(h)
        ox = torch.empty_like(x) if n_obs else None
        check(lib().cut_rhs_jvp(self._h, _ptr(h), n_obs, _ptr(x), _ptr(dh), _ptr(dx), _ptr(oh), _ptr(ox),
                                _stream(stream)))
        return oh, (list(ox) if n_obs else [])

    def rhs_adjoint(self, h, xs, w_h, w_xs, stream=None):
        """Vector-Jacobian product of rhs(): (h_bar, [x_bar_o])."""
        torch = _torch()
        h = _dev_f64(h, self.n, "h", self.device)
        w_h = _dev_f64(w_h, self.n, "w_h", self.device)
        n_obs = len(xs)
        x = torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]) if n_obs else None
        wx = torch.stack([_dev_f64(v, self.n, "w_x", self.device) for v in w_xs]) if n_obs else None
        hb = torch.empty_like(h)
        xb = torch.empty_like(x) if n_obs else None
        check(lib().cut_rhs_adjoint(self._h, _ptr(h), n_obs, _ptr(x), _ptr(w_h), _ptr(wx), _ptr(hb),
                                    _ptr(xb), _stream(stream)))
        return hb, (list(xb) if n_obs else [])

    def _opts(self, method, s0, s1, ds, rtol, atol, max_steps, replay, record_cap):
        o = FlowOpts()
        o.method = RK4 if method == "rk4" else DP45
        o.s0, o.s1, o.ds, o.rtol, o.atol = float(s0), float(s1), float(ds), float(rtol), float(atol)
        o.max_steps = int(max_steps)
        keep = []
        if replay is not None:
            r = np.ascontiguousarray(replay, dtype=np.float64)
            keep.append(r)
            o.replay_steps = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.n_replay = len(r)
        rec = None
        if record_cap:
            rec = np.zeros(record_cap, dtype=np.float64)
            o.record_steps = rec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.record_cap = record_cap
        return o, keep, rec

    def flow(self, h, xs=(), method="rk4", s0=0.0, s1=10.0, ds=1e-3, rtol=1e-10, atol=0.0,
             max_steps=0, replay=None, record_cap=1 << 20, pause_after=0, stream=None):
        """Integrate [h; x_1..] from s0 to s1.  Returns (h, xs, stats, accepted_steps).

        DP45 with pause_after = m stops after m attempts (stats["finished"]
        0); flow(h, xs, s0=stats["s_final"], ds=stats["ds_next"], ...)
        resumes it exactly."""
        torch = _torch()
        h = _dev_f64(h, self.n, "h", self.device).clone()
        n_obs = len(xs)
        x = torch.stack([_dev_f64(v, self.n, "x", self.device) for v in xs]).clone() if n_obs else None
        o, keep, rec = self._opts(method, s0, s1, ds, rtol, atol, max_steps, replay,
                                  record_cap if method == "dp45" else 0)
        o.pause_after = int(pause_after)
        st = FlowStats()
        check(lib().cut_flow(self._h, _ptr(h), n_obs, _ptr(x), ctypes.byref(o), ctypes.byref(st),
                             _stream(stream)))
        stats = {f: getattr(st, f) for f, _ in FlowStats._fields_}
        steps = rec[:min(st.steps, len(rec))].copy() if rec is not None else None
        return h, (list(x) if n_obs else []), stats, steps

    def flow_vjp(self, h0, xs0, yb_h, yb_xs, method="rk4", s0=0.0, s1=10.0, ds=1e-3, steps=None,
                 checkpoint_every=64, stream=None):
        """Discrete adjoint of a flow: dJ/d[h0; x0] given dJ/d[h; x] at s1."""
        torch = _torch()
        h0 = _dev_f64(h0, self.n, "h0", self.device)
        yb_h = _dev_f64(yb_h, self.n, "yb_h", self.device)
        n_obs = len(xs0)
        x0 = torch.stack([_dev_f64(v, self.n, "x0", self.device) for v in xs0]) if n_obs else None
        ybx = torch.stack([_dev_f64(v, self.n, "yb_x", self.device) for v in yb_xs]) if n_obs else None
        gh = torch.empty_like(h0)
        gx = torch.empty_like(x0) if n_obs else None
        o, keep, _ = self._opts(method, s0, s1, ds, 1e-10, 0.0, 0, steps, 0)
        check(lib().cut_flow_vjp(self._h, _ptr(h0), n_obs, _ptr(x0), ctypes.byref(o),
                                 int(checkpoint_every), _ptr(yb_h), _ptr(ybx), _ptr(gh), _ptr(gx),
                                 _stream(stream)))
        return gh, (list(gx) if n_obs else [])

    def flow_batched(self, H, Xs=None, precision="fp64", method="dp45", s0=0.0, s1=10.0, ds=1e-2,
                     rtol=1e-10, atol=0.0, max_steps=0, tile=0, record_cap=0, stream=None):
        """Flows of many coefficient sets through one graph: H [B, n], Xs [B, n_obs, n].

        Returns (H, X, steps, status); with record_cap > 0 also a [B, record_cap]
        FP64 device tensor whose row b holds instance b's accepted step sizes
        (the first steps[b] entries, the rest zero)."""
        torch = _torch()
        H = _dev_f64(H, self.n, "H", self.device).clone()
        B = H.shape[0]
        n_obs = 0 if Xs is None else int(Xs.shape[1])
        X = _dev_f64(Xs, self.n, "X", self.device).clone() if n_obs else None
        steps = torch.zeros(B, dtype=torch.int32, device=self.device)
        status = torch.zeros(B, dtype=torch.int32, device=self.device)
        o, keep, _ = self._opts(method, s0, s1, ds, rtol, atol, max_steps, None, 0)
        rec = None
        if record_cap:
            rec = torch.zeros(B, int(record_cap), dtype=torch.float64, device=self.device)
            o.record_cap = int(record_cap)
            o.batch_record_steps = rec.data_ptr()
        prec = FP64 if precision == "fp64" else FP32REC_FP64STATE
        check(lib().cut_flow_batched(self._h, B, _ptr(H), n_obs, _ptr(X), prec, ctypes.byref(o),
                                     int(tile), _ptr(steps), _ptr(status), _stream(stream)))
        return (H, X, steps, status) if rec is None else (H, X, steps, status, rec)

    @staticmethod
    def last_batched_tile():
        """Tile width this thread's last flow_batched call ran with (0: none)."""
        return int(lib().cut_flow_batched_last_tile())


def ensemble_stats(preds, mask, stream=None):
    """(mean [B, n_out], spread [B]) of K member outputs preds[k] [B, n_out]
    (FP32 device tensors); spread = max over masked outputs of max - min."""
    torch = _torch()
    K = len(preds)
    B, n_out = preds[0].shape
    ps = [p.contiguous() for p in preds]
    arr = (ctypes.c_void_p * K)(*[p.data_ptr() for p in ps])
    mask = torch.as_tensor(mask, dtype=torch.uint8, device=ps[0].device).contiguous()
    mean = torch.empty(B, n_out, dtype=torch.float32, device=ps[0].device)
    spread = torch.empty(B, dtype=torch.float32, device=ps[0].device)
    check(lib().cut_mlp_ensemble_stats(K, B, n_out, arr, _ptr(mask), _ptr(mean), _ptr(spread), _stream(stream)))
    return mean, spread


class MLP:
    """The surrogate network n_in -> H -> H -> n_out (tcgen05 BF16 GEMMs)."""

    def __init__(self, n_in, n_hidden, n_out, seed=0, device=0):
        self._h = VP()
        check(lib().cut_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), int(device),
                                   ctypes.byref(self._h)))
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        self.device_index = int(device)

    @property
    def device(self):
        return _torch().device("cuda", self.device_index)

    def close(self):
        if self._h:
            lib().cut_mlp_free(self._h)
            self._h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_output_affine(self, scale, shift):
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        sh = np.ascontiguousarray(shift, dtype=np.float32)
        check(lib().cut_mlp_set_output_affine(self._h, sc.ctypes.data, sh.ctypes.data))

    def output_affine(self):
        """(scale, shift) of the outputs (host, FP32) as the model uses them."""
        sc = np.empty(self.n_out, dtype=np.float32)
        sh = np.empty(self.n_out, dtype=np.float32)
        check(lib().cut_mlp_get_output_affine(self._h, sc.ctypes.data, sh.ctypes.data))
        return sc, sh

    def set_linear(self, J):
        """Linear skip y += J x (J: [n_out, n_in]); None removes it."""
        if J is None:
            check(lib().cut_mlp_set_linear(self._h, None))
            return
        J = np.ascontiguousarray(J, dtype=np.float32)
        assert J.shape == (self.n_out, self.n_in)
        check(lib().cut_mlp_set_linear(self._h, J.ctypes.data))

    def fit_linear(self, x, t, weight=None, stream=None):
        """Least-squares affine part (shift, J) and residual scale from data
        (x: [B, n_in], t: [B, n_out] FP64), fitted on the device."""
        torch = _torch()
        x = self._f32(x, self.n_in)
        t = t if isinstance(t, torch.Tensor) else torch.as_tensor(np.asarray(t))
        t = t.to(device=self.device, dtype=torch.float64).contiguous()
        assert t.shape == (x.shape[0], self.n_out)
        w = None if weight is None else np.ascontiguousarray(weight, dtype=np.float32)
        check(lib().cut_mlp_fit_linear(self._h, x.shape[0], _ptr(x), _ptr(t),
                                       None if w is None else w.ctypes.data, _stream(stream)))

    def params(self, grads=False):
        out = np.empty(lib().cut_mlp_param_count(self._h), dtype=np.float32)
        check(lib().cut_mlp_get_params(self._h, out.ctypes.data, 1 if grads else 0))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == lib().cut_mlp_param_count(self._h)
        check(lib().cut_mlp_set_params(self._h, flat.ctypes.data))

    def _f32(self, t, cols):
        torch = _torch()
        t = t if isinstance(t, torch.Tensor) else torch.as_tensor(np.asarray(t, dtype=np.float32))
        t = t.to(device=self.device, dtype=torch.float32).contiguous()
        assert t.dim() == 2 and t.shape[1] == cols
        return t

    def forward(self, x, stream=None):
        torch = _torch()
        x = self._f32(x, self.n_in)
        y = torch.empty(x.shape[0], self.n_out, dtype=torch.float32, device=self.device)
        check(lib().cut_mlp_forward(self._h, x.shape[0], _ptr(x), _ptr(y), _stream(stream)))
        return y

    def backward(self, x, target, loss=None, stream=None):
        """Gradients of the standardised MSE; returns the loss tensor (device).

        With ``loss`` (a one-element FP32 device tensor) the batch loss is
        added to it.  Calls that repeat the same x, target and loss buffers
        replay one captured CUDA graph of the whole forward and backward pass."""
        torch = _torch()
        x = self._f32(x, self.n_in)
        t = self._f32(target, self.n_out)
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        check(lib().cut_mlp_backward(self._h, x.shape[0], _ptr(x), _ptr(t), _ptr(loss), _stream(stream)))
        return loss

    def step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        check(lib().cut_mlp_adamw_step(self._h, lr, beta1, beta2, eps, weight_decay, _stream(stream)))

    def status(self):
        check(lib().cut_mlp_status(self._h))

    def inject_stall(self, on):
        """Test hook: make every GEMM's pipeline wait run out (see cut.h)."""
        check(lib().cut_mlp_inject_stall(self._h, 1 if on else 0))

"""Learned surrogate of the flow map theta -> flowed coefficients.

Not in the paper: a screen in front of the graph flow, which stays the
fallback and the judge of the surrogate's error.  Every numerical step runs
in libcut.so: training data come from the batched flow kernel (FP32 records,
FP64 state); the linear part of the map is fitted on the device in FP64
(cut_mlp_fit_linear) and each network learns what it misses with the
library's tcgen05 forward/backward GEMMs and AdamW kernel; rejected queries go
through the FP64 batched flow.

The gate (a reading of "fallback when the error exceeds tol"; the error
estimator is not stated): K networks trained from different initial weights
and data orders answer every query; their spread on the screened
coefficients (max over the coefficients of max - min over the members,
cut_mlp_ensemble_stats) is the error signal, and no flow runs for a query
the gate accepts.  The threshold tau on the spread is calibrated on
validation queries with FP64 flows: the largest tau for which every
validation query with spread <= tau has error <= tol.  The ensemble mean is
the served answer; the other queries fall back to the FP64 flow.
"""
import time

import numpy as np

import paper_2609_14831_b300 as cg


class Surrogate:
    """outputs: the flowed coefficients the networks predict (indices into
    the registry; None = all of them).  Predictions come back as full-length
    vectors with NaN in the coefficients the networks do not predict."""

    def __init__(self, graph, h_ref, P, observables, n_hidden=512, members=2, seed=0, s1=10.0,
                 loose_rtol=1e-6, tight_rtol=1e-10, atol=1e-12, outputs=None):
        import torch
        self.torch = torch
        self.G = graph
        self.dev = graph.device
        self.h_ref = torch.as_tensor(np.asarray(h_ref), dtype=torch.float64, device=self.dev)
        self.P = torch.as_tensor(np.asarray(P), dtype=torch.float64, device=self.dev)
        self.obs = torch.as_tensor(np.stack(observables), dtype=torch.float64, device=self.dev)
        self.n = graph.n
        self.n_in = self.P.shape[1]
        self.s1 = s1
        self.loose_rtol, self.tight_rtol, self.atol = loose_rtol, tight_rtol, atol
        self.outputs = np.arange(self.n) if outputs is None else np.asarray(outputs, dtype=np.int64)
        self._out_dev = torch.as_tensor(self.outputs, device=self.dev)
        self.nets = [cg.MLP(self.n_in, n_hidden, len(self.outputs), seed=seed + 7919 * k,
                            device=graph.device_index) for k in range(members)]
        self.theta_scale = 1.0
        self.tau = None

    def _h0(self, theta):
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float64, device=self.dev)
        return self.h_ref[None, :] + theta @ self.P.T

    def flows(self, theta, precision="fp32", chunk=8192, tile=0):
        """Flowed H for every parameter vector (batched kernel; tile 0 =
        autotuned width, which probes every width on a new batch size)."""
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float64, device=self.dev)
        outs, steps = [], []
        for i in range(0, theta.shape[0], chunk):
            H0 = self._h0(theta[i:i + chunk])
            X0 = self.obs[None].expand(H0.shape[0], -1, -1).contiguous()
            rtol = self.loose_rtol if precision == "fp32" else self.tight_rtol
            atol = 1e-9 if precision == "fp32" else self.atol
            H, _, st, status = self.G.flow_batched(H0, X0, precision=precision, method="dp45", s0=0.0,
                                                   s1=self.s1, ds=1e-2, rtol=rtol, atol=atol, tile=tile)
            if int(status.abs().max().item()) != 0:
                raise cg.CutError(int(status.abs().max().item()), "batched flow failed for some instance")
            outs.append(H)
            steps.append(st)
        return torch.cat(outs), torch.cat(steps)

    def _x(self, theta):
        torch = self.torch
        return (torch.as_tensor(theta, dtype=torch.float32, device=self.dev) / self.theta_scale).contiguous()

    def fit(self, theta, targets, epochs=40, batch=512, lr=2e-3, weight_decay=0.0, seed=0, weight=None, log=None,
            absolute=False):
        """Device least-squares affine part, then AdamW on the standardised
        MSE of each member (library kernels).  targets: [N, n] flowed
        coefficients (the predicted outputs are taken from them).  `weight`
        (per coefficient of the registry, > 0) makes the chosen outputs count
        more in the loss.  absolute: every output's residual is scaled by the
        same constant instead of its own residual RMS, so the loss weighs
        absolute errors (what a gate with an absolute tolerance judges).
        Returns the mean batch loss per epoch of every member."""
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float32, device=self.dev)
        targets = torch.as_tensor(targets, dtype=torch.float64, device=self.dev)
        targets = targets.index_select(1, self._out_dev).contiguous()
        self.theta_scale = float(theta.abs().max().item()) or 1.0
        x = (theta / self.theta_scale).contiguous()
        t32 = targets.float()
        N = x.shape[0]
        steps = max(1, N // batch)
        total = epochs * steps
        w = None if weight is None else np.asarray(weight, dtype=np.float64)[self.outputs]
        hists = []
        for k, net in enumerate(self.nets):
            if absolute:
                # residual RMS of each output (the scale of an unweighted fit),
                # then weights that bring every scale to their median
                net.fit_linear(x, targets, None)
                rms = net.output_affine()[0].astype(np.float64)
                wa = (rms / np.median(rms)) ** 2
                net.fit_linear(x, targets, wa if w is None else w * wa)
            else:
                net.fit_linear(x, targets, w)
            g = torch.Generator(device="cpu").manual_seed(seed + 104729 * k)
            # fixed staging buffers: every step reuses the same device pointers,
            # so the library replays its captured forward/backward graph
            xs = torch.empty(min(batch, N), x.shape[1], dtype=torch.float32, device=self.dev)
            ts = torch.empty(min(batch, N), t32.shape[1], dtype=torch.float32, device=self.dev)
            loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
            hist, it = [], 0
            for ep in range(epochs):
                perm = torch.randperm(N, generator=g).to(self.dev)
                loss.zero_()
                for s in range(steps):
                    idx = perm[s * batch:(s + 1) * batch]
                    torch.index_select(x, 0, idx, out=xs)
                    torch.index_select(t32, 0, idx, out=ts)
                    cur = lr * 0.5 * (1 + np.cos(np.pi * it / total))   # cosine decay
                    net.backward(xs, ts, loss=loss)
                    net.step(lr=cur, weight_decay=weight_decay)
                    it += 1
                hist.append(float(loss.item()) / steps)
                if log:
                    log(k, ep, hist[-1])
            net.status()
            hists.append(hist)
        return hists

    def predict_members(self, theta):
        x = self._x(theta)
        return [net.forward(x) for net in self.nets]

    def predict(self, theta, screened_idx=None):
        """(ensemble mean [B, n] FP64, NaN where not predicted; spread [B]
        over the screened coefficients, which must be predicted ones)."""
        torch = self.torch
        preds = self.predict_members(theta)
        screened = self.outputs if screened_idx is None else np.asarray(screened_idx)
        mask = np.isin(self.outputs, screened).astype(np.uint8)
        assert int(mask.sum()) == len(np.unique(screened)), "screened coefficients must be predicted outputs"
        mean, spread = cg.ensemble_stats(preds, mask)
        if len(self.outputs) == self.n and np.array_equal(self.outputs, np.arange(self.n)):
            return mean.double(), spread
        full = torch.full((mean.shape[0], self.n), float("nan"), dtype=torch.float64, device=self.dev)
        full.index_copy_(1, self._out_dev, mean.double())
        return full, spread

    def calibrate(self, theta, exact, screened_idx, tol):
        """tau = the largest spread for which every validation query with a
        spread no larger has error <= tol on the screened outputs (-1: none)."""
        torch = self.torch
        mean, spread = self.predict(theta, screened_idx)
        idx = torch.as_tensor(np.asarray(screened_idx), device=self.dev)
        err = (mean[:, idx] - exact[:, idx]).abs().max(dim=1).values.cpu().numpy()
        sp = spread.cpu().numpy().astype(np.float64)
        order = np.argsort(sp, kind="stable")
        worst = np.maximum.accumulate(err[order])
        ok = np.nonzero(worst <= tol)[0]
        self.tau = float(sp[order[ok[-1]]]) if ok.size else -1.0
        return self.tau, float(np.mean(sp <= self.tau))

    @staticmethod
    def fallback_tile(count, sms=148):
        """Tile width of the batched fallback for `count` queries: the
        narrowest tile whose CTAs still fit on the SMs.  A CTA streams every
        record for each of its TILE slots at once, so its step costs about
        TILE / 32 warp instructions per record and a narrower tile finishes
        a small batch sooner; 8 (the width the autotuner picks for full
        batches) once the narrower ones would need more CTAs than SMs."""
        for t in (2, 4):
            if count <= t * sms:
                return t
        return 8

    def fallback(self, theta):
        """FP64 flows of the rejected queries.  A batched flow's wall time is
        set by its longest instance run on few SMs, so a handful of queries
        is faster through the single-instance flow (all SMs on one
        instance); larger sets take the batched kernel at a fixed tile
        width chosen from their count (no autotuning inside a served call)."""
        torch = self.torch
        theta = np.asarray(theta)
        if len(theta) > self.plain_max:
            H0 = self._h0(theta)
            X0 = self.obs[None].expand(H0.shape[0], -1, -1).contiguous()
            H, _, _, status = self.G.flow_batched(H0, X0, precision="fp64", method="dp45", s0=0.0, s1=self.s1,
                                                  ds=1e-2, rtol=self.tight_rtol, atol=self.atol,
                                                  tile=self.fallback_tile(len(theta)))
            if int(status.abs().max().item()) != 0:
                raise cg.CutError(int(status.abs().max().item()), "fallback flow failed")
            return H
        H0 = self._h0(theta)
        outs = []
        for b in range(len(theta)):
            h, _, _, _ = self.G.flow(H0[b], list(self.obs), method="dp45", s0=0.0, s1=self.s1, ds=1e-2,
                                     rtol=self.tight_rtol, atol=self.atol)
            outs.append(h)
        return torch.stack(outs)

    # 8-orbital model, DP45 to s = 10, rtol 1e-10, one B300: the plain flow
    # takes 38 ms per query; the batched fallback 0.58 s for up to 296
    # queries at tile 2, 1.07 s up to 592 at tile 4, 2.04 s for 1024 at tile 8
    plain_max = 15

    def warm_up(self):
        """Load every kernel a served call may launch (the network, the plain
        flow and the batched flow at each fallback tile width) on a short
        span, so that no served call pays for first use."""
        torch = self.torch
        th = np.zeros((2, self.n_in))
        self.predict(th, self.outputs[:1])
        H0 = self._h0(th)
        X0 = self.obs[None].expand(H0.shape[0], -1, -1).contiguous()
        for t in (2, 4, 8):
            self.G.flow_batched(H0, X0, precision="fp64", method="dp45", s0=0.0, s1=0.02, ds=1e-2,
                                rtol=self.tight_rtol, atol=self.atol, tile=t)
        self.G.flow(H0[0], list(self.obs), method="dp45", s0=0.0, s1=0.02, ds=1e-2, rtol=self.tight_rtol,
                    atol=self.atol)
        torch.cuda.synchronize()

    def screen(self, theta, screened_idx):
        """Served answers: the ensemble mean where the spread is <= tau, the
        FP64 flow elsewhere.  Returns (H, accepted mask (numpy), timings)."""
        torch = self.torch
        assert self.tau is not None, "calibrate() first"
        theta = np.asarray(theta)
        t0 = time.perf_counter()
        mean, spread = self.predict(theta, screened_idx)
        ok = spread.cpu().numpy().astype(np.float64) <= self.tau
        t1 = time.perf_counter()
        rej = np.nonzero(~ok)[0]
        if rej.size:
            mean[torch.as_tensor(rej, device=self.dev)] = self.fallback(theta[rej])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return mean, ok, {"predict_s": t1 - t0, "fallback_s": t2 - t1, "accepted": int(ok.sum()),
                          "queries": int(ok.size)}

    def rank_screen(self, theta, coef, frac):
        """Rank queries by the ensemble's predicted coefficient `coef` and
        flow (FP64) only the best-ranked `frac` of them: returns (indices of
        the flowed queries, their exact coefficient, seconds, timings)."""
        torch = self.torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mean, _ = self.predict(theta, [coef])
        # the ranking of one coefficient on the host: a torch sort would load
        # its sort kernels on first use (seconds) inside a served call
        order = np.argsort(mean[:, coef].cpu().numpy(), kind="stable")
        chosen = np.sort(order[: int(frac * len(order))])
        t1 = time.perf_counter()
        th = theta[chosen] if isinstance(theta, np.ndarray) else theta[torch.as_tensor(chosen, device=self.dev)]
        exact, _ = self.flows(th, "fp64", tile=self.fallback_tile(len(th)))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return chosen, exact[:, coef], t2 - t0, {"rank_s": t1 - t0, "flow_s": t2 - t1, "flowed": int(len(chosen))}

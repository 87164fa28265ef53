"""Learned surrogate of the flow map theta -> flowed coefficients.

Not in the paper: a warm start and screen in front of the graph flow, which
stays the fallback and the judge of the surrogate's error.  Every numerical
step runs in libcut.so: training data come from the batched flow kernel
(FP32 records, FP64 state), the network is trained by the library's tcgen05
forward/backward GEMMs and AdamW kernel, and rejected queries go through the
FP64 batched flow.

Screening rule (a reading of "fallback when the error exceeds tol"): each
query is flowed once with the loose FP32 batched flow; if the network's
prediction of any screened coefficient differs from it by more than `tol`,
the query falls back to the full FP64 flow, otherwise the prediction is used.
"""
import time

import numpy as np

import paper_2609_14831_b300 as cg


class Surrogate:
    def __init__(self, graph, h_ref, P, observables, n_hidden=512, seed=0, s1=10.0,
                 loose_rtol=1e-6, tight_rtol=1e-10, atol=1e-12):
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
        self.net = cg.MLP(self.n_in, n_hidden, self.n, seed=seed, device=graph.device_index)
        self.theta_scale = 1.0

    def _h0(self, theta):
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float64, device=self.dev)
        return self.h_ref[None, :] + theta @ self.P.T

    def flows(self, theta, precision="fp32", chunk=8192):
        """Flowed H for every parameter vector (batched kernel)."""
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float64, device=self.dev)
        outs, steps = [], []
        for i in range(0, theta.shape[0], chunk):
            H0 = self._h0(theta[i:i + chunk])
            X0 = self.obs[None].expand(H0.shape[0], -1, -1).contiguous()
            rtol = self.loose_rtol if precision == "fp32" else self.tight_rtol
            atol = 1e-9 if precision == "fp32" else self.atol
            H, _, st, status = self.G.flow_batched(H0, X0, precision=precision, method="dp45", s0=0.0,
                                                   s1=self.s1, ds=1e-2, rtol=rtol, atol=atol)
            if int(status.abs().max().item()) != 0:
                raise cg.CutError(int(status.abs().max().item()), "batched flow failed for some instance")
            outs.append(H)
            steps.append(st)
        return torch.cat(outs), torch.cat(steps)

    def fit(self, theta, targets, epochs=40, batch=512, lr=2e-3, weight_decay=0.0, seed=0, log=None):
        """Standardise the targets, then AdamW on the MSE (library kernels)."""
        torch = self.torch
        theta = torch.as_tensor(theta, dtype=torch.float32, device=self.dev)
        targets = torch.as_tensor(targets, dtype=torch.float64, device=self.dev)
        self.theta_scale = float(theta.abs().max().item()) or 1.0
        x = (theta / self.theta_scale).contiguous()
        # linear part by least squares (FP64), the network learns the rest
        A = torch.cat([torch.ones(x.shape[0], 1, dtype=torch.float64, device=self.dev), x.double()], dim=1)
        coef = torch.linalg.lstsq(A, targets).solution               # [1 + n_in, n]
        mu, J = coef[0], coef[1:].T.contiguous()
        resid = targets - A @ coef
        sd = resid.std(0).clamp_min(1e-9)
        self.mu, self.sd, self.J = mu, sd, J
        self.net.set_output_affine(sd.float().cpu().numpy(), mu.float().cpu().numpy())
        self.net.set_linear(J.float().cpu().numpy())
        t32 = targets.float()
        g = torch.Generator(device="cpu").manual_seed(seed)
        N = x.shape[0]
        steps = max(1, N // batch)
        total = epochs * steps
        hist = []
        it = 0
        # fixed staging buffers: every step reuses the same device pointers, so
        # the library replays its captured forward/backward graph
        xs = torch.empty(min(batch, N), x.shape[1], dtype=torch.float32, device=self.dev)
        ts = torch.empty(min(batch, N), t32.shape[1], dtype=torch.float32, device=self.dev)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        for ep in range(epochs):
            perm = torch.randperm(N, generator=g).to(self.dev)
            loss.zero_()
            for s in range(steps):
                idx = perm[s * batch:(s + 1) * batch]
                torch.index_select(x, 0, idx, out=xs)
                torch.index_select(t32, 0, idx, out=ts)
                # cosine learning-rate decay
                cur = lr * 0.5 * (1 + np.cos(np.pi * it / total))
                self.net.backward(xs, ts, loss=loss)
                self.net.step(lr=cur, weight_decay=weight_decay)
                it += 1
            hist.append(float(loss.item()) / steps)   # mean batch loss of the epoch
            if log:
                log(ep, hist[-1])
        self.net.status()
        return hist

    def predict(self, theta):
        torch = self.torch
        x = (torch.as_tensor(theta, dtype=torch.float32, device=self.dev) / self.theta_scale).contiguous()
        return self.net.forward(x).double()

    def screen(self, theta, screened_idx, tol=1e-4):
        """Surrogate + fallback.  Returns (H, used_network mask, timings)."""
        torch = self.torch
        t0 = time.perf_counter()
        pred = self.predict(theta)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loose, _ = self.flows(theta, "fp32")
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        idx = torch.as_tensor(screened_idx, device=self.dev)
        err = (pred[:, idx] - loose[:, idx]).abs().max(dim=1).values
        ok = err <= tol
        out = pred.clone()
        rej = torch.nonzero(~ok).flatten()
        if rej.numel():
            tight, _ = self.flows(theta[rej.cpu().numpy()] if isinstance(theta, np.ndarray) else theta[rej], "fp64")
            out[rej] = tight
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        return out, ok, {"predict_s": t1 - t0, "loose_s": t2 - t1, "fallback_s": t3 - t2,
                         "accepted": int(ok.sum().item()), "queries": int(ok.numel())}

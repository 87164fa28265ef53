"""torch.autograd bridge: a flow whose backward is the library's discrete
adjoint (paper Sec. 2.4: reverse propagation through the same stored records;
Eq. directional-derivative for the generator variation).

The forward runs cut_flow and keeps the accepted step sizes; the backward
runs cut_flow_vjp over exactly those steps, with forward states stored every
`checkpoint_every` steps and recomputed in between.
"""
import torch


class _Flow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h0, x0, graph, opts, checkpoint_every):
        xs = list(x0) if x0 is not None and x0.numel() else []
        hs, xo, stats, steps = graph.flow(h0, xs, **opts)
        ctx.graph, ctx.opts, ctx.every = graph, dict(opts), checkpoint_every
        ctx.steps = steps
        ctx.stats = stats
        ctx.has_x = bool(xs)
        ctx.save_for_backward(h0, x0 if x0 is not None else torch.empty(0, device=h0.device))
        xout = torch.stack(xo) if xo else torch.empty(0, graph.n, dtype=h0.dtype, device=h0.device)
        return hs, xout

    @staticmethod
    def backward(ctx, gh, gx):
        h0, x0 = ctx.saved_tensors
        o = ctx.opts
        xs = list(x0) if ctx.has_x else []
        if gh is None:
            gh = torch.zeros_like(h0)
        gxs = [] if not ctx.has_x else list(gx if gx is not None else torch.zeros_like(x0))
        gh0, gx0 = ctx.graph.flow_vjp(h0, xs, gh, gxs, method=o.get("method", "rk4"), s0=o.get("s0", 0.0),
                                      s1=o.get("s1", 10.0), ds=o.get("ds", 1e-3),
                                      steps=ctx.steps if o.get("method") == "dp45" else None,
                                      checkpoint_every=ctx.every)
        return gh0, (torch.stack(gx0) if ctx.has_x else None), None, None, None


def flow(graph, h0, x0=None, checkpoint_every=64, **opts):
    """Differentiable flow: returns (h(s1), x(s1)); gradients reach h0 and x0."""
    return _Flow.apply(h0, x0, graph, opts, checkpoint_every)

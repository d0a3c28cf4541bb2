"""torch.autograd.Function over the C ABI: the value V(x, t) of every query point
as a differentiable function of the query points x, the cost weights W, the
cost centre c and the dynamics parameters.

forward  = hj_solve_batch (trajectories kept for the backward pass)
backward = hj_solve_grad  (adjoint="envelope": the adjoint of the value at the
           converged saddle, envelope theorem on Eq. (disclaxBE)), or
           hj_solve_grad_unrolled (adjoint="unrolled": reverse sweep through the
           iterations each point ran, checkpointed every `checkpoint_every`)
"""
import torch

from . import binding


class HJValue(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xq, t, W, c, dyn, family, N, opts_kw):
        opts_kw = dict(opts_kw)
        adjoint = opts_kw.pop("adjoint", "envelope")
        ckpt = opts_kw.pop("checkpoint_every", 32)
        d = xq.shape[1]
        prob = binding.Problem(family, d, dyn.detach().cpu().numpy(), W.detach().cpu().numpy(),
                               c.detach().cpu().numpy())
        opts = binding.make_opts(**opts_kw)
        out = binding.solve_batch(prob, xq.detach().to(torch.float64).contiguous(),
                                  t.detach().to(torch.float64).contiguous(), N, opts,
                                  return_traj=True)
        ctx.prob, ctx.N, ctx.precision = prob, N, opts_kw.get("precision", "fp32")
        ctx.dyn_shape = dyn.shape
        ctx.devices = (W.device, c.device, dyn.device)
        ctx.adjoint, ctx.ckpt, ctx.opts = adjoint, ckpt, opts
        ctx.save_for_backward(t, out["traj_x"], out["traj_p"], xq.detach().to(torch.float64),
                              out["iters"])
        ctx.mark_non_differentiable(out["iters"], out["status"])
        return out["V"], out["iters"], out["status"]

    @staticmethod
    def backward(ctx, gV, _gi, _gs):
        t, tx, tp, xq, iters = ctx.saved_tensors
        if ctx.adjoint == "unrolled":
            g = binding.solve_grad_unrolled(ctx.prob, xq, t.to(torch.float64), ctx.N, ctx.opts,
                                            iters, gV.to(torch.float64).contiguous(),
                                            checkpoint_every=ctx.ckpt)
        else:
            g = binding.solve_grad(ctx.prob, t.to(torch.float64), ctx.N, ctx.precision, tx, tp,
                                   gV.to(torch.float64).contiguous(),
                                   want_dxq=ctx.needs_input_grad[0])
        dW_dev, dc_dev, dyn_dev = ctx.devices
        ddyn = g["ddyn"].reshape(ctx.dyn_shape).to(dyn_dev) if g["ddyn"].numel() else None
        return (g["dxq"], None, g["dW"].to(dW_dev), g["dc"].to(dc_dev), ddyn, None, None, None)


def hj_value(xq, t, W, c, dyn, *, family, N, **opts_kw):
    """V [B] (differentiable in xq, W, c, dyn), iters [B], status [B].
    opts_kw: sigma, tau, tol, max_iter, check_every, precision, seed, ... as
    binding.make_opts, plus adjoint ("envelope" | "unrolled") and
    checkpoint_every.  W, c, dyn may live on any device (copied to the solver)."""
    if dyn is None:
        dyn = torch.zeros(0, dtype=torch.float64)
    return HJValue.apply(xq, t, W, c, dyn, family, int(N), dict(opts_kw))

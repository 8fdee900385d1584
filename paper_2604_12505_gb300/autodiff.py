"""Differentiable rollout of the SPH step (the linearizations of Section 5.2).

``rollout(params, xv0, body0, u)`` runs K steps of one tank from the fluid
state xv0 [N, 4], the body state body0 [6] and the inputs u [K, 3] and
returns the sampled outputs y [n_samples, 11].  It is a
``torch.autograd.Function`` with hand-written derivatives from the library:

* reverse mode (``backward``): the adjoint sweep ``sph_vjp``, which runs the
  K steps forward keeping a checkpoint every ``checkpoint_every`` steps, then
  recomputes each segment and steps the adjoint kernels back through it.  It
  gives the gradients with respect to xv0, body0 and u;
* forward mode (``torch.autograd.forward_ad``): the tangent kernels
  ``sph_jvp``.

Both freeze the neighbour set of each step, as the derivatives of Section 5.2
are taken along a trajectory.
"""
from __future__ import annotations

import torch

from .sph import Sim


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, body0, xv0, params, checkpoint_every):
        ctx.meta = [(t.device, t.dtype) for t in (u, body0, xv0)]
        u = u.detach().to("cuda", torch.float64).contiguous()
        b0 = body0.detach().to("cuda", torch.float64).reshape(1, 6).contiguous()
        x0 = xv0.detach().to("cuda", torch.float32).contiguous()
        K = int(u.shape[0])
        with Sim(params) as sim:
            sim.set_state(x0, b0)
            y = sim.step(K, u=u[None])
            sim.check()
        ctx.params, ctx.K, ctx.C = params, K, int(checkpoint_every)
        ctx.state0 = (x0, b0, u)
        return y[0]

    @staticmethod
    def backward(ctx, gy):
        x0, b0, u = ctx.state0
        with Sim(ctx.params) as sim:
            sim.set_state(x0, b0)
            xb, bb, ub = sim.vjp(ctx.K, u=u[None], ybar=gy.to("cuda", torch.float64)[None],
                                 checkpoint_every=ctx.C)
            sim.check()
        (du, tu), (db, tb), (dx, tx) = ctx.meta
        return ub[0].to(du, tu), bb[0].to(db, tb), xb.to(dx, tx), None, None

    @staticmethod
    def jvp(ctx, du, dbody0, dxv0, _dparams, _dc):
        x0, b0, u = ctx.state0
        K = ctx.K
        du = torch.zeros((K, 3), dtype=torch.float64, device="cuda") if du is None else du.to("cuda", torch.float64)
        db = torch.zeros(6, dtype=torch.float64, device="cuda") if dbody0 is None else dbody0.to("cuda", torch.float64)
        dx = None if dxv0 is None else dxv0.to("cuda", torch.float32).contiguous()
        with Sim(ctx.params) as sim:
            sim.set_state(x0, b0)
            _, dy, _, _ = sim.jvp(K, u=u[None], du=du.reshape(1, K, 3).contiguous(), dxv0=dx,
                                  dbody0=db.reshape(1, 6).contiguous())
            sim.check()
        return dy[0]


def rollout(params: dict, xv0, body0, u, checkpoint_every: int = 10):
    """Sampled outputs [ceil(K / outer_every), 11] of K steps of one tank
    (float64, CUDA), differentiable with respect to u [K, 3], body0 [6] and
    the fluid state xv0 [N, 4] (rows x, y, vx, vy in builder order)."""
    if not torch.is_tensor(xv0):
        xv0 = torch.as_tensor(xv0, dtype=torch.float32)
    if not torch.is_tensor(body0):
        body0 = torch.as_tensor(body0, dtype=torch.float64)
    if not torch.is_tensor(u):
        u = torch.as_tensor(u, dtype=torch.float64)
    return _Rollout.apply(u, body0, xv0, params, checkpoint_every)

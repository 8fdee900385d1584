"""Differentiable rollout of the SPH step (the linearizations of Section 5.2).

``rollout(params, xv0, body0, u)`` runs K steps of one tank from the fluid
state xv0 and the body state body0 under the inputs u and returns the sampled
outputs y [n_samples, 11]; it is a ``torch.autograd.Function`` whose
derivatives with respect to u [K, 3] and body0 [6] come from the library's
hand-written forward-mode derivative (``sph_jvp``: tangent kernels along the
FP32 trajectory with the neighbour set of each step frozen):

* forward mode (``torch.func.jvp`` / ``torch.autograd.forward_ad``): one
  tangent rollout from the start of the window;
* reverse mode (``backward``): the Jacobian columns of the low-dimensional
  inputs, computed as one batched tangent rollout per checkpoint, each column
  a copy of the tank in the batch (a batch reproduces single-tank runs bit for
  bit).  The forward pass stores the state every ``checkpoint_every`` steps;
  the columns of u_k start from the checkpoint at or before step k, since u_k
  cannot affect earlier samples.  The gradient is then J^T g.

The fluid state xv0 is an input without a gradient here (its Jacobian has
4 N columns); its tangent is available through ``Sim.jvp``.
"""
from __future__ import annotations

import torch

from .sph import Sim


def _as_dev(t, dtype):
    return torch.as_tensor(t, dtype=dtype).to("cuda").contiguous()


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, body0, params, xv0, checkpoint_every):
        K = int(u.shape[0])
        outer = int(params["outer_every"])
        C = int(checkpoint_every)
        if C <= 0 or C % outer:
            raise ValueError("checkpoint_every must be a positive multiple of outer_every")
        ctx.u_meta = (u.device, u.dtype)
        ctx.b_meta = (body0.device, body0.dtype)
        u = u.detach().to("cuda", torch.float64).contiguous()
        b0 = body0.detach().to("cuda", torch.float64).reshape(1, 6).contiguous()
        ckpts = []
        ys = []
        with Sim(params) as sim:
            sim.set_state(xv0, b0)
            for c0 in range(0, K, C):
                ckpts.append(tuple(t.clone() for t in sim.state()))
                n = min(C, K - c0)
                ys.append(sim.step(n, u=u[c0:c0 + n][None].contiguous()))
            sim.check()
        ctx.params, ctx.C, ctx.K, ctx.outer = params, C, K, outer
        ctx.ckpts = ckpts
        ctx.u_dev = u
        return torch.cat(ys, dim=1)[0]

    @staticmethod
    def backward(ctx, gy):
        u, C, K, outer, params = ctx.u_dev, ctx.C, ctx.K, ctx.outer, ctx.params
        gy = gy.to("cuda", torch.float64)
        gu = torch.zeros((K, 3), dtype=torch.float64, device="cuda")
        gb = torch.zeros(6, dtype=torch.float64, device="cuda")
        for g, (xv_c, body_c) in enumerate(ctx.ckpts):
            c0 = g * C
            n_u = min(C, K - c0)
            ncol = 3 * n_u + (6 if g == 0 else 0)
            Kg = K - c0
            du = torch.zeros((ncol, Kg, 3), dtype=torch.float64, device="cuda")
            db = torch.zeros((ncol, 6), dtype=torch.float64, device="cuda")
            j = torch.arange(3 * n_u, device="cuda")
            du[j, j // 3, j % 3] = 1.0
            if g == 0:
                db[3 * n_u + torch.arange(6, device="cuda"), torch.arange(6, device="cuda")] = 1.0
            with Sim([params] * ncol) as bs:
                bs.set_state(xv_c.repeat(ncol, 1), body_c.repeat(ncol, 1))
                _, dy, _, _ = bs.jvp(Kg, u=u[c0:][None].expand(ncol, Kg, 3).contiguous(), du=du, dbody0=db)
                bs.check()
            s0 = c0 // outer
            contrib = torch.einsum("bsj,sj->b", dy, gy[s0:s0 + dy.shape[1]])
            gu[c0:c0 + n_u] = contrib[:3 * n_u].reshape(n_u, 3)
            if g == 0:
                gb = contrib[3 * n_u:]
        return (gu.to(*ctx.u_meta), gb.reshape(6).to(*ctx.b_meta), None, None, None)

    @staticmethod
    def jvp(ctx, du, dbody0, _dparams, _dxv0, _dc):
        K = ctx.K
        du = torch.zeros((K, 3), dtype=torch.float64, device="cuda") if du is None else du.to("cuda", torch.float64)
        db = torch.zeros(6, dtype=torch.float64, device="cuda") if dbody0 is None else dbody0.to("cuda", torch.float64)
        xv_c, body_c = ctx.ckpts[0]
        with Sim(ctx.params) as sim:
            sim.set_state(xv_c, body_c)
            _, dy, _, _ = sim.jvp(K, u=ctx.u_dev[None], du=du.reshape(1, K, 3).contiguous(),
                                  dbody0=db.reshape(1, 6).contiguous())
            sim.check()
        return dy[0]


def rollout(params: dict, xv0, body0, u, checkpoint_every: int = 10):
    """Sampled outputs [ceil(K / outer_every), 11] of K steps of one tank
    (float64, CUDA), differentiable with respect to u [K, 3] and body0 [6]."""
    xv0 = _as_dev(xv0, torch.float32)
    return _Rollout.apply(u, body0, params, xv0, checkpoint_every)

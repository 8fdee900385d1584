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


# ---------------------------------------------------------------------------
# Linearization of the dynamics (Section 5.2): the Jacobian of xdot = f(x, u)
# and its eigenvalues along a trajectory
# ---------------------------------------------------------------------------
def state_index(n_f: int) -> dict:
    """Layout of the state vector x (n = 4 n_f + 6): the fluid state flattened
    row-major (x, y, vx, vy per particle, in the order of Sim.state), then the
    body (r_x, r_y, theta, rdot_x, rdot_y, thetadot).  Returns the indices of
    the positions and of their velocities, pairwise."""
    fl = torch.arange(4 * n_f).reshape(n_f, 4)
    pos = torch.cat([fl[:, :2].reshape(-1), 4 * n_f + torch.arange(3)])
    vel = torch.cat([fl[:, 2:].reshape(-1), 4 * n_f + 3 + torch.arange(3)])
    return dict(n=4 * n_f + 6, pos=pos, vel=vel)


def jacobian(params: dict, xv, body, u=None, block: int = 256) -> torch.Tensor:
    """A = df/dx [n, n] (float64, CUDA) of the continuous dynamics
    xdot = f(x, u) of one tank at the state (xv [N, 4], body [6]) and input
    u [3], open loop, in the layout of state_index.  The position rows are the
    identity on the velocity columns; the velocity rows come from
    Jacobian-vector products (Sim.eval_jvp) of a batch of ``block`` copies of
    the tank, copy i carrying the unit tangent of one column."""
    xv = torch.as_tensor(xv, dtype=torch.float32).reshape(-1, 4).cuda()
    body = torch.as_tensor(body, dtype=torch.float64).reshape(6).cuda()
    n_f = xv.shape[0]
    ix = state_index(n_f)
    n = ix["n"]
    u1 = None if u is None else torch.as_tensor(u, dtype=torch.float64).reshape(1, 3).cuda()
    nb = max(1, min(block, n))
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    A[ix["pos"].cuda(), ix["vel"].cuda()] = 1.0
    vel_f = torch.arange(4 * n_f, device="cuda").reshape(n_f, 4)[:, 2:].reshape(-1)
    with Sim([params] * nb) as sim:
        sim.set_state(xv.repeat(nb, 1), body.repeat(nb, 1))
        for c0 in range(0, n, nb):
            cols = torch.arange(c0, min(c0 + nb, n), device="cuda")
            k = cols.numel()
            dxv = torch.zeros((nb, n_f * 4), dtype=torch.float32, device="cuda")
            db = torch.zeros((nb, 6), dtype=torch.float64, device="cuda")
            fl = cols < 4 * n_f
            rows = torch.arange(k, device="cuda")
            dxv[rows[fl], cols[fl]] = 1.0
            db[rows[~fl], cols[~fl] - 4 * n_f] = 1.0
            dacc, dba = sim.eval_jvp(dxv.reshape(nb * n_f, 4), db, u=None if u1 is None else u1.repeat(nb, 1))
            sim.check()
            A[vel_f, c0:c0 + k] = dacc.reshape(nb, 2 * n_f)[:k].T.double()
            A[4 * n_f + 3:, c0:c0 + k] = dba[:k, 3:].T
    return A


def eigenvalues_over_time(params: dict, xv0, body0, u, at_steps, block: int = 256):
    """Eigenvalues of A = df/dx at the given step indices of the open-loop
    trajectory from (xv0, body0) under the inputs u [K, 3].  Returns a list of
    complex [n] tensors (CPU)."""
    at = sorted(int(k) for k in at_steps)
    u = torch.as_tensor(u, dtype=torch.float64).reshape(-1, 3).cuda()
    out = []
    with Sim(params) as sim:
        sim.set_state(torch.as_tensor(xv0, dtype=torch.float32), torch.as_tensor(body0, dtype=torch.float64))
        k = 0
        for ka in at:
            if ka > k:
                sim.step(ka - k, u=u[k:ka][None], record=False)
                k = ka
            xv, body = sim.state()
            sim.check()
            A = jacobian(params, xv, body[0], u[ka] if ka < u.shape[0] else None, block=block)
            out.append(torch.linalg.eigvals(A.cpu()))  # host LAPACK (a dense nonsymmetric eigensolver)
    return out

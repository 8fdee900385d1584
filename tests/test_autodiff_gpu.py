"""GPU tests of the differentiable rollout (paper_2604_12505_gb300/autodiff.py):
the rollout equals plain stepping, forward mode equals the library's tangent
rollout, reverse mode (the adjoint sweep) is its transpose, and the gradient
with respect to inputs, body and fluid state matches central finite
differences of the FP64 oracle."""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu
CFG = dict(W.SMALL, outer_every=5)
K = 40


def _setup(orc):
    xv, x, v, gB, p = oracle_state(orc, CFG, 0.1, 0.2, seed=4)
    body = np.array([0.002, -0.001, 0.05, 0.01, 0.0, 0.2])
    u = W.bang_bang_slew(K, CFG["dt"], tau=400.0, t1=K * CFG["dt"] / 2)
    u[:, 0], u[:, 1] = 150.0, -90.0
    return xv, x, v, gB, p, body, u


def test_rollout_equals_plain_stepping(orc):
    torch = need_gpu()
    from paper_2604_12505_gb300.autodiff import rollout
    from paper_2604_12505_gb300.sph import Sim
    xv, _, _, _, _, body, u = _setup(orc)
    y = rollout(CFG, xv, torch.tensor(body), torch.tensor(u), checkpoint_every=10)
    with Sim(CFG) as s:
        s.set_state(xv, body)
        y1 = s.step(K, u=u[None])[0]
    assert torch.equal(y, y1)


def test_forward_mode_equals_tangent_rollout_and_reverse_mode_is_its_transpose(orc):
    torch = need_gpu()
    import torch.autograd.forward_ad as fwAD
    from paper_2604_12505_gb300.autodiff import rollout
    from paper_2604_12505_gb300.sph import Sim
    xv, _, _, _, _, body, u = _setup(orc)
    rng = np.random.default_rng(11)
    vu = rng.normal(size=(K, 3)) * np.array([20.0, 20.0, 2.0])
    vb = rng.normal(size=6) * np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2])
    vx = np.concatenate([rng.normal(0, 1e-3, (xv.shape[0], 2)), rng.normal(0, 1e-2, (xv.shape[0], 2))], axis=1)
    U, B0 = torch.tensor(u, device="cuda"), torch.tensor(body, device="cuda")
    X0 = torch.tensor(xv, device="cuda")
    VU, VB = torch.tensor(vu, device="cuda"), torch.tensor(vb, device="cuda")
    VX = torch.tensor(vx, dtype=torch.float32, device="cuda")
    with fwAD.dual_level():
        yd = rollout(CFG, fwAD.make_dual(X0, VX), fwAD.make_dual(B0, VB), fwAD.make_dual(U, VU))
        jv = fwAD.unpack_dual(yd).tangent
    with Sim(CFG) as s:
        s.set_state(xv, body)
        _, dy, _, _ = s.jvp(K, u=u[None], du=vu[None], dxv0=vx.astype(np.float32), dbody0=vb[None])
    assert torch.equal(jv, dy[0])
    # <J v, w> = <v, J^T w>, with J^T w from the adjoint sweep
    w = torch.tensor(rng.normal(size=tuple(jv.shape)), device="cuda")
    U.requires_grad_(True)
    B0.requires_grad_(True)
    X0.requires_grad_(True)
    y = rollout(CFG, X0, B0, U, checkpoint_every=10)
    gu, gb, gx = torch.autograd.grad(y, (U, B0, X0), grad_outputs=w)
    lhs = float((jv * w).sum())
    rhs = float((gu * VU).sum() + (gb * VB).sum() + (gx.double() * VX.double()).sum())
    assert rhs == pytest.approx(lhs, rel=1e-4)


def test_gradient_matches_oracle_finite_differences(orc):
    torch = need_gpu()
    from paper_2604_12505_gb300.autodiff import rollout
    xv, x, v, gB, p, body, u = _setup(orc)
    rng = np.random.default_rng(12)
    U = torch.tensor(u, device="cuda", requires_grad=True)
    B0 = torch.tensor(body, device="cuda", requires_grad=True)
    X0 = torch.tensor(xv, device="cuda", requires_grad=True)
    y = rollout(CFG, X0, B0, U, checkpoint_every=10)
    w = rng.normal(size=tuple(y.shape))
    gu, gb, gx = torch.autograd.grad(y, (U, B0, X0), grad_outputs=torch.tensor(w, device="cuda"))
    eps = 1e-4
    for k in range(3):
        du = rng.normal(size=(K, 3)) * np.array([20.0, 20.0, 2.0])
        db = rng.normal(size=6) * np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2])
        dxv = np.concatenate([rng.normal(0, 1e-3, (x.shape[0], 2)), rng.normal(0, 1e-2, (x.shape[0], 2))], axis=1)
        ys = []
        for sgn in (1.0, -1.0):
            ys.append(orc.run(p, x + sgn * eps * dxv[:, :2], v + sgn * eps * dxv[:, 2:], gB, body + sgn * eps * db, K,
                              u=u + sgn * eps * du)[3])
        fd = (ys[0] - ys[1]) / (2 * eps)
        lhs = float(np.sum(w * fd))
        rhs = float((gu.cpu().numpy() * du).sum() + (gb.cpu().numpy() * db).sum() +
                    (gx.cpu().numpy().astype(np.float64) * dxv).sum())
        tol = 2e-3 * np.abs(w * fd).sum()
        assert abs(rhs - lhs) <= tol, (k, lhs, rhs, tol)

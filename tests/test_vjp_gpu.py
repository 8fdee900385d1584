"""GPU reverse-mode derivative (sph_vjp) of K SPH steps.

The adjoint must be the transpose of the tangent map sph_jvp carries: for any
directions v = (dxv0, dbody0, du) and w = (ybar, xvbar_K, bodybar_K),
<J v, w> = <v, J^T w> up to FP32 rounding of the two different evaluation
orders (1e-4 of the summed magnitudes).  It is also checked against central
finite differences of the FP64 oracle (2e-3, the tangent test's tolerance),
and must not depend on the checkpoint interval or on batching.
"""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _setup(orc, cfg, K, seed=4):
    xv, x, v, gB, p = oracle_state(orc, cfg, 0.1, 0.2, seed=seed)
    body = np.array([0.002, -0.001, 0.05, 0.01, 0.0, 0.2])
    u = W.bang_bang_slew(K, cfg["dt"], tau=400.0, t1=K * cfg["dt"] / 2)
    u[:, 0], u[:, 1] = 150.0, -90.0
    return xv, x, v, gB, p, body, u


def _dirs(rng, n, K, ns):
    dxv = np.concatenate([rng.normal(0, 1e-3, (n, 2)), rng.normal(0, 1e-2, (n, 2))], axis=1)
    db = rng.normal(0, 1.0, 6) * np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2])
    du = rng.normal(0, 1.0, (K, 3)) * np.array([20.0, 20.0, 2.0])
    yb = rng.normal(size=(ns, 11))
    xb = rng.normal(size=(n, 4))
    bb = rng.normal(size=6)
    return dxv, db, du, yb, xb, bb


def _inner_pairs(sim, xv, body, u, K, v, w):
    dxv, db, du = v
    yb, xb, bb = w
    sim.set_state(xv, body)
    _, dy, dxvK, dbK = sim.jvp(K, u=u[None], du=du[None], dxv0=dxv.astype(np.float32), dbody0=db[None])
    lhs_terms = np.concatenate([(dy.cpu().numpy()[0] * yb).ravel(), (dxvK.cpu().numpy() * xb).ravel(),
                                dbK.cpu().numpy()[0] * bb])
    sim.set_state(xv, body)
    xb0, bb0, ub = sim.vjp(K, u=u[None], ybar=yb[None], xvbar=xb.astype(np.float32), bodybar=bb[None])
    rhs_terms = np.concatenate([(xb0.cpu().numpy().astype(np.float64) * dxv).ravel(), bb0.cpu().numpy()[0] * db,
                                (ub.cpu().numpy()[0] * du).ravel()])
    return lhs_terms, rhs_terms, (xb0, bb0, ub)


@pytest.mark.parametrize("cfg,K", [(dict(W.SMALL, outer_every=5), 30), (dict(W.JVP, outer_every=10), 20),
                                   (dict(W.SMALL, outer_every=5, n_rings=1, ghost_spacing=0.9, gamma1=0.5,
                                         ghost_pressure_clamp=1), 30)])
def test_adjoint_is_the_transpose_of_the_tangent_map(orc, cfg, K):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    xv, x, v, gB, p, body, u = _setup(orc, cfg, K)
    rng = np.random.default_rng(30)
    with Sim(cfg) as s:
        ns = s.samples_for(K)
        for _ in range(3):
            dxv, db, du, yb, xb, bb = _dirs(rng, xv.shape[0], K, ns)
            lt, rt, _ = _inner_pairs(s, xv, body, u, K, (dxv, db, du), (yb, xb, bb))
            s.check()
            scale = max(np.abs(lt).sum(), np.abs(rt).sum())
            assert abs(lt.sum() - rt.sum()) <= 1e-4 * scale, (lt.sum(), rt.sum(), scale)


def test_adjoint_of_each_part_separately(orc):
    # one input direction against one output direction at a time: u -> samples,
    # body -> final fluid, fluid -> final body
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg, K = dict(W.SMALL, outer_every=5), 25
    xv, x, v, gB, p, body, u = _setup(orc, cfg, K, seed=6)
    rng = np.random.default_rng(31)
    n = xv.shape[0]
    with Sim(cfg) as s:
        ns = s.samples_for(K)
        dxv, db, du, yb, xb, bb = _dirs(rng, n, K, ns)
        z = np.zeros
        cases = [((z((n, 4)), z(6), du), (yb, z((n, 4)), z(6))),
                 ((z((n, 4)), db, z((K, 3))), (z((ns, 11)), xb, z(6))),
                 ((dxv, z(6), z((K, 3))), (z((ns, 11)), z((n, 4)), bb))]
        for vv, ww in cases:
            lt, rt, _ = _inner_pairs(s, xv, body, u, K, vv, ww)
            scale = max(np.abs(lt).sum(), np.abs(rt).sum())
            assert scale > 0
            assert abs(lt.sum() - rt.sum()) <= 1e-4 * scale, (lt.sum(), rt.sum(), scale)


def test_adjoint_does_not_depend_on_checkpoints_or_batching(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg, K = dict(W.SMALL, outer_every=5), 25
    xv, x, v, gB, p, body, u = _setup(orc, cfg, K, seed=7)
    rng = np.random.default_rng(32)
    outs = []
    with Sim(cfg) as s:
        ns = s.samples_for(K)
        _, _, _, yb, xb, bb = _dirs(rng, xv.shape[0], K, ns)
        for C in (1, 7, 25):
            s.set_state(xv, body)
            r = s.vjp(K, u=u[None], ybar=yb[None], xvbar=xb.astype(np.float32), bodybar=bb[None], checkpoint_every=C)
            outs.append([t.cpu().numpy() for t in r])
            state = [t.cpu().numpy() for t in s.state()]
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            np.testing.assert_array_equal(a, b)
    # the simulator is left at state K
    with Sim(cfg) as s:
        s.set_state(xv, body)
        s.step(K, u=u[None])
        ref = [t.cpu().numpy() for t in s.state()]
    np.testing.assert_array_equal(state[0], ref[0])
    np.testing.assert_array_equal(state[1], ref[1])
    # a batch of two copies gives each copy's adjoint
    with Sim([cfg, cfg]) as sb:
        sb.set_state(np.concatenate([xv, xv]), np.stack([body, body]))
        r = sb.vjp(K, u=np.stack([u, u]), ybar=np.stack([yb, yb]), xvbar=np.concatenate([xb, xb]).astype(np.float32),
                   bodybar=np.stack([bb, bb]))
        xb0, bb0, ub = [t.cpu().numpy() for t in r]
    n = xv.shape[0]
    np.testing.assert_array_equal(xb0[:n], outs[0][0])
    np.testing.assert_array_equal(xb0[n:], outs[0][0])
    np.testing.assert_array_equal(bb0[1], outs[0][1][0])
    np.testing.assert_array_equal(ub[1], outs[0][2][0])


def test_adjoint_matches_oracle_finite_differences(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg, K = dict(W.SMALL, outer_every=5), 30
    xv, x, v, gB, p, body, u = _setup(orc, cfg, K, seed=8)
    rng = np.random.default_rng(33)
    n = xv.shape[0]
    with Sim(cfg) as s:
        ns = s.samples_for(K)
        _, _, _, yb, xb, bb = _dirs(rng, n, K, ns)
        s.set_state(xv, body)
        xb0, bb0, ub = [t.cpu().numpy().astype(np.float64) for t in
                        s.vjp(K, u=u[None], ybar=yb[None], xvbar=xb.astype(np.float32), bodybar=bb[None])]
    eps = 1e-4
    for k in range(3):
        dxv, db, du, _, _, _ = _dirs(rng, n, K, ns)
        outs = []
        for sgn in (1.0, -1.0):
            xr, vr, br, yr, _ = orc.run(p, x + sgn * eps * dxv[:, :2], v + sgn * eps * dxv[:, 2:], gB,
                                        body + sgn * eps * db, K, u=u + sgn * eps * du)
            outs.append((np.concatenate([xr, vr], axis=1), br, yr))
        fd_xv = (outs[0][0] - outs[1][0]) / (2 * eps)
        fd_b = (outs[0][1] - outs[1][1]) / (2 * eps)
        fd_y = (outs[0][2] - outs[1][2]) / (2 * eps)
        terms_fd = np.concatenate([(fd_y * yb).ravel(), (fd_xv * xb).ravel(), fd_b * bb])
        rhs = (xb0 * dxv).sum() + (bb0[0] * db).sum() + (ub[0] * du).sum()
        scale = np.abs(terms_fd).sum()
        assert abs(rhs - terms_fd.sum()) <= 2e-3 * scale, (k, terms_fd.sum(), rhs, scale)

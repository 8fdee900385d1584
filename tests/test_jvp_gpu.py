"""GPU forward-mode derivative (sph_jvp) against central finite differences of
the FP64 oracle.

For a seeded direction (dx0, dv0, dbody0, du) over a window of K steps:
    FD = (y(x0 + e d, u + e du) - y(x0 - e d, u - e du)) / (2 e)
computed by the oracle in FP64, against the tangent the GPU carries along
its FP32 trajectory.  The tangent's error comes from FP32 arithmetic over K
steps and from linearizing along the FP32 rather than the FP64 trajectory;
the tolerance below is 2e-3 of the largest tangent entry of each group.
"""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import TRAJ_GROUPS, need_gpu, oracle_state

pytestmark = pytest.mark.gpu
TOL = 2e-3


def _direction(n, K, seed):
    rng = np.random.default_rng(seed)
    dxv = np.concatenate([rng.normal(0, 1e-3, (n, 2)), rng.normal(0, 1e-2, (n, 2))], axis=1)
    db = rng.normal(0, 1.0, 6) * np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2])
    du = rng.normal(0, 1.0, (K, 3)) * np.array([20.0, 20.0, 2.0])
    return dxv, db, du


def _fd(orc, p, x, v, gB, body, u, d, K, eps):
    dxv, db, du = d
    outs = []
    for sgn in (1.0, -1.0):
        xr, vr, br, yr, _ = orc.run(p, x + sgn * eps * dxv[:, :2], v + sgn * eps * dxv[:, 2:], gB,
                                    body + sgn * eps * db, K, u=u + sgn * eps * du)
        outs.append((xr, vr, br, yr))
    (xa, va, ba, ya), (xb, vb, bb, yb) = outs
    return (ya - yb) / (2 * eps), (np.concatenate([xa - xb, va - vb], axis=1)) / (2 * eps), (ba - bb) / (2 * eps)


@pytest.mark.parametrize("cfg,K,n_dir", [(dict(W.SMALL, outer_every=5), 50, 8), (dict(W.JVP, outer_every=10), 50, 2)])
def test_jvp_matches_oracle_finite_differences(orc, cfg, K, n_dir):
    torch = need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    xv, x, v, gB, p = oracle_state(orc, cfg, 0.1, 0.2, seed=4)
    body = np.array([0.002, -0.001, 0.05, 0.01, 0.0, 0.2])
    u = W.bang_bang_slew(K, cfg["dt"], tau=400.0, t1=K * cfg["dt"] / 2)
    u[:, 0], u[:, 1] = 150.0, -90.0
    eps = 1e-4
    with Sim(cfg) as s:
        for k in range(n_dir):
            d = _direction(x.shape[0], K, seed=100 + k)
            dy_fd, dxv_fd, db_fd = _fd(orc, p, x, v, gB, body, u, d, K, eps)
            s.set_state(xv, body)
            y, dy, dxv, db = s.jvp(K, u=u[None], du=d[2][None], dxv0=d[0].astype(np.float32), dbody0=d[1][None])
            s.check()
            dy = dy.cpu().numpy()[0]
            dxv = dxv.cpu().numpy().astype(np.float64)
            db = db.cpu().numpy()[0]
            for name, cols in dict(TRAJ_GROUPS, force=[6, 7], torque=[8]).items():
                den = np.linalg.norm(dy_fd[:, cols], axis=1).max()
                err = np.linalg.norm(dy[:, cols] - dy_fd[:, cols], axis=1).max() / den
                assert err <= TOL, (k, name, err)
            for blk in (slice(0, 2), slice(2, 4)):
                den = np.linalg.norm(dxv_fd[:, blk], axis=1).max()
                assert np.linalg.norm(dxv[:, blk] - dxv_fd[:, blk], axis=1).max() <= TOL * den
            assert np.abs(db - db_fd).max() <= TOL * np.abs(db_fd).max()


def test_jvp_primal_equals_step_and_zero_tangent(orc):
    torch = need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg = dict(W.SMALL, outer_every=5)
    xv, *_ = oracle_state(orc, cfg, 0.1, 0.2, seed=5)
    K = 40
    u = W.bang_bang_slew(K, cfg["dt"], tau=300.0, t1=K * cfg["dt"] / 2)
    with Sim(cfg) as s:
        s.set_tile(3)
        s.set_state(xv, np.zeros(6))
        y0 = s.step(K, u=u[None]).cpu().numpy()
        x0 = s.state()[0].cpu().numpy()
        s.set_state(xv, np.zeros(6))
        y1, dy, dxv, db = [t.cpu().numpy() for t in s.jvp(K, u=u[None])]
        x1 = s.state()[0].cpu().numpy()
        s.check()
    np.testing.assert_allclose(y1, y0, rtol=0, atol=1e-9 * np.abs(y0).max())
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-6)
    assert np.all(dy == 0) and np.all(dxv == 0) and np.all(db == 0)

"""Derivatives as the differentiation workload states them: the 15,532-particle
tank (R = 0.5 m, 50 % fill, dx = 0.005 m), windows of K = 50 steps along the
slew, 8 seeded directions drawn from N(0, I) over the whole input
(x, v, body, u) and normalised (seed 7), central differences of the FP64
oracle with eps = 1e-6 ||(x0, v0, body0, u)||, checkpoints every 10 steps
for the adjoint.

Tolerance: 2e-3 of the largest entry of each output group.  The GPU tangent
and adjoint run in FP32 along the FP32 trajectory; the central difference of
the FP64 oracle is exact to O(eps^2) away from the switches of Algorithm 1.
For every direction the oracle reports how many pairs take a switch
differently between the two ends of the difference: a crossing of a kernel
support (where Eqs. 22 and 23 vanish with two continuous derivatives, so
the step map stays smooth) or of the min(., 0) of Eq. 18 (a kink).  Those
counts are printed with the error of the direction, and the tolerance holds
for every direction, flagged or not.
"""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import TRAJ_GROUPS, need_gpu, oracle_state

pytestmark = pytest.mark.gpu
TOL = 2e-3
K = 50
CFG = dict(W.JVP, outer_every=10)


@pytest.fixture(scope="module")
def setup(orc):
    need_gpu()
    xv, x, v, gB, p = oracle_state(orc, CFG, 0.1, 0.2, seed=4)
    body = np.array([0.002, -0.001, 0.05, 0.01, 0.0, 0.2])
    u = W.bang_bang_slew(K, CFG["dt"], tau=2.0, t1=0.5)
    norm = np.sqrt((x ** 2).sum() + (v ** 2).sum() + (body ** 2).sum() + (u ** 2).sum())
    return dict(xv=xv, x=x, v=v, gB=gB, p=p, body=body, u=u, eps=1e-6 * norm)


def _directions(n, seed=7, count=8):
    """N(0, I) over (dx, dv) [n, 4], dbody [6], du [K, 3], normalised."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dxv, db, du = rng.normal(size=(n, 4)), rng.normal(size=6), rng.normal(size=(K, 3))
        s = np.sqrt((dxv ** 2).sum() + (db ** 2).sum() + (du ** 2).sum())
        out.append((dxv / s, db / s, du / s))
    return out


def _ends(S, d):
    dxv, db, du = d
    e = S["eps"]
    return [((S["x"] + g * e * dxv[:, :2], S["v"] + g * e * dxv[:, 2:], S["body"] + g * e * db), S["u"] + g * e * du)
            for g in (1.0, -1.0)]


def _fd(orc, S, d):
    outs = []
    for (x, v, b), u in _ends(S, d):
        xr, vr, br, yr, _ = orc.run(S["p"], x, v, S["gB"], b, K, u=u)
        outs.append((np.concatenate([xr, vr], axis=1), br, yr))
    e2 = 2 * S["eps"]
    return (outs[0][2] - outs[1][2]) / e2, (outs[0][0] - outs[1][0]) / e2, (outs[0][1] - outs[1][1]) / e2


def _crossings(orc, S, d):
    ends = _ends(S, d)
    return orc.switches_cross(S["p"], S["gB"], [e[0] for e in ends], [e[1] for e in ends])


def test_tangent_against_oracle_differences(orc, setup):
    from paper_2604_12505_gb300.sph import Sim
    S = setup
    report = []
    with Sim(CFG) as s:
        for k, d in enumerate(_directions(S["x"].shape[0])):
            dy_fd, dxv_fd, db_fd = _fd(orc, S, d)
            s.set_state(S["xv"], S["body"])
            _, dy, dxv, db = s.jvp(K, u=S["u"][None], du=d[2][None], dxv0=d[0].astype(np.float32),
                                    dbody0=d[1][None])
            s.check()
            dy = dy.cpu().numpy()[0]
            dxv = dxv.cpu().numpy().astype(np.float64)
            db = db.cpu().numpy()[0]
            errs = {}
            for name, cols in dict(TRAJ_GROUPS, force=[6, 7], torque=[8]).items():
                den = np.linalg.norm(dy_fd[:, cols], axis=1).max()
                errs[name] = np.linalg.norm(dy[:, cols] - dy_fd[:, cols], axis=1).max() / den
            for name, blk in (("dx", slice(0, 2)), ("dv", slice(2, 4))):
                den = np.linalg.norm(dxv_fd[:, blk], axis=1).max()
                errs[name] = np.linalg.norm(dxv[:, blk] - dxv_fd[:, blk], axis=1).max() / den
            errs["dbody"] = np.abs(db - db_fd).max() / np.abs(db_fd).max()
            cr = _crossings(orc, S, d)
            report.append((k, max(errs.values()), cr))
            print(f"direction {k}: max error {max(errs.values()):.2e}; switches crossed within +-eps: "
                  f"support {cr['support']}, clip {cr['clip']} (first at step {cr['first']})")
            assert max(errs.values()) <= TOL, (k, errs, cr)
    assert len(report) == 8


def test_adjoint_against_oracle_differences(orc, setup):
    # <v, J^T w> from the reverse sweep (checkpoints every 10 steps) against
    # <J v, w> from the oracle's central differences, for 3 of the directions.
    from paper_2604_12505_gb300.sph import Sim
    S = setup
    n = S["x"].shape[0]
    rng = np.random.default_rng(71)
    with Sim(CFG) as s:
        ns = s.samples_for(K)
        yb = rng.normal(size=(ns, 11))
        xb = rng.normal(size=(n, 4)) * 1e-3
        bb = rng.normal(size=6)
        s.set_state(S["xv"], S["body"])
        xb0, bb0, ub = [t.cpu().numpy().astype(np.float64) for t in
                        s.vjp(K, u=S["u"][None], ybar=yb[None], xvbar=xb.astype(np.float32), bodybar=bb[None],
                              checkpoint_every=10)]
        s.check()
    for k, d in enumerate(_directions(n)[:3]):
        dy_fd, dxv_fd, db_fd = _fd(orc, S, d)
        terms = np.concatenate([(dy_fd * yb).ravel(), (dxv_fd * xb).ravel(), db_fd * bb])
        rhs = (xb0 * d[0]).sum() + (bb0[0] * d[1]).sum() + (ub[0] * d[2]).sum()
        scale = np.abs(terms).sum()
        print(f"adjoint direction {k}: |<v, J^T w> - <J v, w>| / sum|terms| = {abs(rhs - terms.sum()) / scale:.2e}")
        assert abs(rhs - terms.sum()) <= TOL * scale, (k, terms.sum(), rhs, scale)

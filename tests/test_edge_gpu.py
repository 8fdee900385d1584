"""Edge cases of the C ABI on the GPU: empty and full tanks, ragged batches,
cell-capacity overflow, zero-step calls, rejected arguments, and surrogate
shapes other than the default one."""
import numpy as np
import pytest

from oracle import lpv as L
from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def test_empty_tank_moves_as_a_rigid_body(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfg = dict(W.SMALL, fill=0.0)
    p = orc.params(**cfg)
    assert orc.tank_counts(p)[0] == 0
    n = 200
    u = W.piecewise_profile(n, cfg["dt"], seed=3, hold=(0.001, 0.003))
    ref = np.repeat([0.05, -0.02], n // 2 // cfg["outer_every"])
    body0 = np.array([0.01, -0.02, 0.1, 0.001, -0.002, 0.05])
    with Sim(cfg) as s:
        assert s.n_fluid == [0]
        xv = np.zeros((0, 4), dtype=np.float32)
        s.set_state(xv, body0)
        y = s.step(n, u=u[None], ctrl=dict(omega=0.2 * np.pi, xi=0.7), theta_ref=ref[None]).cpu().numpy()[0]
        s.check()
    _, gB = orc.tank(p)
    yo = orc.run(p, np.zeros((0, 2)), np.zeros((0, 2)), gB, body0, n, u=u, theta_ref=ref, use_ctrl=True)[3]
    np.testing.assert_allclose(y[:, :6], yo[:, :6], rtol=1e-12, atol=1e-15)
    assert np.all(y[:, 6:] == 0.0)


def test_ragged_batch_with_empty_and_full_tanks(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    cfgs = [dict(W.SMALL, fill=0.0), W.TINY, dict(W.SMALL, fill=1.0), dict(W.TINY, fill=0.3)]
    counts = [orc.tank_counts(orc.params(**c))[0] for c in cfgs]
    assert counts[0] == 0 and counts[2] > counts[1] > counts[3] > 0
    n = 40
    us = [W.piecewise_profile(n, c["dt"], seed=70 + i, hold=(0.0005, 0.001)) for i, c in enumerate(cfgs)]
    singles = []
    for c, u in zip(cfgs, us):
        with Sim(c) as s:
            singles.append(s.step(n, u=u[None]).cpu().numpy()[0])
    with Sim(cfgs) as sb:
        assert sb.n_fluid == counts
        yb = sb.step(n, u=np.stack(us)).cpu().numpy()
        sb.check()
    for i in range(len(cfgs)):
        np.testing.assert_array_equal(yb[i], singles[i])


def test_cell_overflow_is_reported_not_written_out_of_bounds(orc):
    need_gpu()
    from paper_2604_12505_gb300 import _lib
    from paper_2604_12505_gb300.sph import Sim
    cfg = W.TINY
    xv, *_ = oracle_state(orc, cfg)
    crowd = xv.copy()
    crowd[:80, :2] = crowd[0, :2]          # 80 particles in one cell of capacity 32
    crowd[:80, 0] += np.linspace(0, 1e-4, 80, dtype=np.float32)
    with Sim(cfg) as s:
        s.set_state(crowd, np.zeros(6))
        assert s.check(raise_on_error=False, reset=True) & _lib.FLAG_CELL_FULL
        s.set_state(xv, np.zeros(6))
        s.step(5)
        assert s.check() == 0


def test_zero_steps_leave_the_state_unchanged(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    xv, *_ = oracle_state(orc, W.SMALL, 0.1, 0.1, seed=5)
    with Sim(W.SMALL) as s:
        s.set_state(xv, np.zeros(6))
        before = [t.cpu().numpy() for t in s.state()]
        y = s.step(0)
        assert y.shape[1] == 0
        after = [t.cpu().numpy() for t in s.state()]
        np.testing.assert_array_equal(before[0], after[0])
        np.testing.assert_array_equal(before[1], after[1])


@pytest.mark.parametrize("bad", [dict(dx=0.0), dict(fill=1.5), dict(R=-0.5), dict(dx=0.6)])
def test_invalid_tank_parameters_are_rejected(bad):
    need_gpu()
    from paper_2604_12505_gb300 import _lib
    from paper_2604_12505_gb300.sph import Sim
    with pytest.raises(_lib.SphError) as ei:
        Sim(dict(W.SMALL, **bad))
    assert ei.value.code == -1


def test_surrogate_of_other_dimensions_matches_oracle():
    # n_x = 9 (na = 3, n_y = 3), n_u = 2, one scheduling variable; ragged trajectory count
    need_gpu()
    from paper_2604_12505_gb300.lpv import Model
    nx, nu, ny, n_p = 9, 2, 3, 1
    rng = np.random.default_rng(20)
    W0 = np.zeros((nx + ny, (1 + n_p) * (nx + nu)))
    for i in range(1 + n_p):
        A = rng.normal(size=(nx, nx))
        A *= (0.6 if i == 0 else 0.2) / np.linalg.norm(A, 2)
        blk = slice(i * (nx + nu), (i + 1) * (nx + nu))
        W0[:nx, blk] = np.concatenate([A, 0.3 * rng.normal(size=(nx, nu))], axis=1)
        W0[nx:, blk][:, :nx] = 0.3 * rng.normal(size=(ny, nx))
    n, T = 21, 33
    u = rng.normal(size=(n, T, nu))
    p = rng.uniform(-1, 1, size=(n, T, n_p))
    y = rng.normal(size=(n, T, ny))
    m = Model(dict(n_x=nx, n_u=nu, n_y=ny, n_p=n_p, na=3, sigma2=1e-3))
    scales = np.concatenate([np.ones(nu + ny), np.zeros(n_p), np.ones(n_p), np.full(n_p, -np.inf),
                             np.full(n_p, np.inf)]).astype(np.float32)
    m.set_params(W0.reshape(nx + ny, 1 + n_p, nx + nu).transpose(1, 0, 2), scales)
    W32 = m.get_params()[0].transpose(1, 0, 2).reshape(nx + ny, -1).astype(np.float64)
    loss, g = m.loss_grad(u, y, p)
    assert loss == pytest.approx(L.loss(W32, list(u), list(y), list(p), nx, 1e-3), rel=1e-4)
    go = L.loss_grad(W32, list(u), list(y), list(p), nx, 1e-3, mask=L.d_mask(nx, nu, ny, n_p))
    g = g.transpose(1, 0, 2).reshape(nx + ny, -1)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    yg = m.predict(u, p).cpu().numpy()
    for b in (0, 7, 20):
        yo, _ = L.simulate(W32, u[b], p[b], nx)
        assert np.abs(yg[b] - yo).max() <= 1e-3 * np.abs(yo).max()


def test_single_trajectory_of_one_sample():
    need_gpu()
    from paper_2604_12505_gb300.lpv import Model
    rng = np.random.default_rng(21)
    m = Model(dict(n_p=0, sigma2=0.0))
    W0 = 0.2 * rng.normal(size=m.shape_W)
    W0[0, 12:, 12:] = 0.0
    m.set_params(W0, np.ones(m.n_scales, dtype=np.float32))
    u = rng.normal(size=(1, 1, 3))
    y = rng.normal(size=(1, 1, 4))
    loss, g = m.loss_grad(u, y, np.zeros((1, 1, 0)))
    # x_0 = 0 and D = 0: the first output is 0 whatever W is, and no weight acts on it
    assert loss == pytest.approx(float((y ** 2).sum()), rel=1e-6)
    assert np.all(g == 0.0)


@pytest.mark.parametrize("cfg", [dict(n_x=13, n_u=3), dict(n_y=2, n_x=4, na=2), dict(n_p=3), dict(n_x=10, na=3)])
def test_unsupported_surrogate_shapes_are_rejected(cfg):
    need_gpu()
    from paper_2604_12505_gb300 import _lib
    from paper_2604_12505_gb300.lpv import Model
    with pytest.raises(_lib.SphError):
        Model(cfg)


def test_lti_closed_loop_matches_oracle():
    need_gpu()
    from paper_2604_12505_gb300.lpv import Model
    rng = np.random.default_rng(22)
    nx = 12
    m = Model(dict(n_p=0))
    A = rng.normal(size=(nx, nx))
    A *= 0.7 / np.linalg.norm(A, 2)
    Wt = np.zeros((16, 15))
    Wt[:nx, :nx] = A
    Wt[:nx, nx:] = 0.05 * rng.normal(size=(nx, 3))
    Wt[nx:, :nx] = 0.05 * rng.normal(size=(4, nx))
    scales = np.array([20.0, 20.0, 2.0, 30.0, 30.0, 3.0, 0.05], dtype=np.float32)
    m.set_params(Wt[None], scales)
    W32 = m.get_params()[0][0].astype(np.float64)
    B, T = 5, 120
    F = rng.uniform(-20, 20, size=(B, T, 2))
    tau = rng.uniform(-2, 2, size=(B, T))
    ref = np.repeat(rng.uniform(-0.1, 0.1, size=(B, T // 20)), 20, axis=1)
    fill = rng.uniform(0.2, 0.8, size=B)
    body = dict(m=500.0, J=50.0, Ts=0.005, n_sub=10, ctrl_omega=0.2 * np.pi, ctrl_xi=0.7)
    out = m.simulate(F, tau, ref, fill, body).cpu().numpy()
    sc = dict(u=scales[:3].astype(np.float64), y=scales[3:7].astype(np.float64), p_mean=np.zeros(0), p_scale=np.ones(0))
    for b in range(B):
        o = L.closed_loop(W32, nx, sc, body, fill[b], F[b], tau[b], ref[b], body["Ts"], body["n_sub"],
                          dict(omega=body["ctrl_omega"], xi=body["ctrl_xi"]))
        for cols in ([0, 1], [2], [3, 4], [5]):
            den = np.linalg.norm(o[:, cols], axis=1).max()
            assert np.linalg.norm(out[b][:, cols] - o[:, cols], axis=1).max() <= 1e-3 * den

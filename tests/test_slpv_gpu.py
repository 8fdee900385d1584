"""GPU parity of the self-scheduled LPV surrogate (Section 4, Section 5.3.2)
against the FP64 oracle, through the C ABI of include/slpv.h.

Tolerances: the kernels run in FP32 with the parameters and data rounded to
FP32; loss relative 1e-4; gradient, free run and closed loop within 1e-3 of
the largest entry of the oracle's result.
"""
import numpy as np
import pytest

from oracle import slpv as S
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

NU = NY = 3


def _theta(nx, seed, m1=0.1):
    rng = np.random.default_rng(seed)
    P = {
        "M0": rng.normal(0, 0.3, (nx + NY, nx + NU)),
        "M1": rng.normal(0, m1, (nx + NY, nx + NU)),
        "W1": rng.normal(0, 0.5, (4, nx + NU)),
        "b1": rng.normal(0, 0.1, 4),
        "W2": rng.normal(0, 0.5, (4, 4)),
        "b2": rng.normal(0, 0.1, 4),
        "w3": rng.normal(0, 0.5, 4),
        "b3": rng.normal(0, 0.1, 1),
    }
    P["M0"][:nx, :nx] *= 0.5
    th = (S.pack(P) * S.d_mask(nx, NU, NY)).astype(np.float32)
    return th.astype(np.float64), th


def _data(n, T, seed, scales):
    rng = np.random.default_rng(seed)
    u = (rng.normal(size=(n, T, 3)) * scales[:3]).astype(np.float32)
    y = (rng.normal(size=(n, T, 3)) * scales[3:]).astype(np.float32)
    return u, y


@pytest.mark.parametrize("nx", [4, 2])
def test_loss_and_gradient_match_oracle(nx):
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    th64, th32 = _theta(nx, 1)
    u, y = _data(3, 60, 2, sc)
    U = [u[i].astype(np.float64) / sc[:3] for i in range(3)]
    Y = [y[i].astype(np.float64) / sc[3:] for i in range(3)]
    sigma2 = 1e-3
    ref_l = S.loss(th64, U, Y, nx, sigma2)
    ref_g = S.loss_grad(th64, U, Y, nx, sigma2, S.d_mask(nx, NU, NY))
    m = VelocityModel(nx=nx, sigma2=sigma2)
    m.set_params(th32, sc)
    loss, g = m.loss_grad(torch.tensor(u), torch.tensor(y))
    l2, g2 = m.loss_grad(torch.tensor(u), torch.tensor(y))
    loss, g = float(loss.item()), g.cpu().numpy()
    assert abs(loss - ref_l) <= 1e-4 * ref_l
    assert np.abs(g - ref_g).max() <= 1e-3 * np.abs(ref_g).max()
    assert float(l2.item()) == loss and np.array_equal(g2.cpu().numpy(), g)  # fixed-order sums
    mask = S.d_mask(nx, NU, NY)
    assert np.all(g[mask == 0] == 0)
    # the LTI stage trains M_0 only, the scheduling stage everything else
    nm = (nx + NY) * (nx + NU)
    _, gl = m.loss_grad(torch.tensor(u), torch.tensor(y), stage=m.LTI)
    gl = gl.cpu().numpy()
    assert np.all(gl[nm:] == 0) and np.array_equal(gl[:nm], g[:nm])
    _, gs = m.loss_grad(torch.tensor(u), torch.tensor(y), stage=m.SCHEDULING)
    gs = gs.cpu().numpy()
    assert np.all(gs[:nm] == 0) and np.array_equal(gs[nm:], g[nm:])
    m.close()


def test_free_run_and_augmentation_match_oracle():
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([10.0, 10.0, 1.0, 0.2, 0.2, 0.1], dtype=np.float32)
    th64, th32 = _theta(4, 3)
    u, _ = _data(5, 80, 4, sc)
    m = VelocityModel(nx=4)
    m.set_params(th32, sc)
    vel, pos = m.predict(torch.tensor(u), Ts=0.05)
    vel, pos = vel.cpu().numpy(), pos.cpu().numpy()
    for i in range(5):
        e, yh = S.augment(th64, u[i].astype(np.float64) / sc[:3], 4, 3, 0.05)
        rv, rp = yh * sc[3:], e * sc[3:]
        assert np.abs(vel[i] - rv).max() <= 1e-3 * np.abs(rv).max()
        assert np.abs(pos[i] - rp).max() <= 1e-3 * np.abs(rp).max()
    m.close()


def test_closed_loop_matches_oracle():
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    from paper_2604_12505_gb300 import workloads as W
    sc = np.array([20.0, 20.0, 2.0, 0.05, 0.05, 0.02], dtype=np.float32)
    th64, th32 = _theta(4, 5, m1=0.2)
    B, T, Ts = 6, 120, 0.05
    F = np.stack([W.piecewise_profile(T, Ts, seed=40 + b)[:, :2] for b in range(B)])
    tau = np.stack([W.piecewise_profile(T, Ts, seed=60 + b)[:, 2] for b in range(B)])
    ref = np.stack([W.theta_ref_steps(T, Ts, seed=80 + b) for b in range(B)])
    pd = dict(J=133.84, omega=0.2 * np.pi, xi=0.7)
    m = VelocityModel(nx=4)
    m.set_params(th32, sc)
    out = m.simulate(F, tau, ref, Ts, pd["J"], pd["omega"], pd["xi"]).cpu().numpy()
    for b in range(B):
        r = S.closed_loop(th64, 4, dict(u=sc[:3].astype(np.float64), y=sc[3:].astype(np.float64)), F[b], tau[b],
                          ref[b], Ts, pd)
        for blk in (slice(0, 3), slice(3, 6)):
            assert np.abs(out[b][:, blk] - r[:, blk]).max() <= 1e-3 * np.abs(r[:, blk]).max()
    m.close()


def test_normalize_gives_channel_rms():
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    u, y = _data(7, 50, 9, np.array([3.0, 1.0, 0.5, 2.0, 0.1, 0.01], dtype=np.float32))
    m = VelocityModel(nx=4)
    m.normalize(torch.tensor(u), torch.tensor(y))
    _, sc = m.get_params()
    ref = np.sqrt(np.concatenate([(u.astype(np.float64) ** 2).mean(axis=(0, 1)),
                                  (y.astype(np.float64) ** 2).mean(axis=(0, 1))]))
    np.testing.assert_allclose(sc, ref, rtol=1e-6)
    m.close()


def test_first_adam_step_and_training_descends():
    """Adam's first step moves every trained entry by lr against the sign of
    its gradient; training from a random model lowers the loss."""
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    th64, th32 = _theta(4, 11, m1=0.05)
    # data from a teacher model, so a good fit exists
    teacher = _theta(4, 12, m1=0.1)[1]
    u, _ = _data(16, 100, 13, sc)
    mt = VelocityModel(nx=4)
    mt.set_params(teacher, sc)
    y, _ = mt.predict(torch.tensor(u), Ts=0.05)
    mt.close()
    m = VelocityModel(nx=4, sigma2=1e-6)
    m.set_params(th32, sc)
    _, g = m.loss_grad(torch.tensor(u), y)
    g = g.cpu().numpy()
    # an iteration evaluates its iterate and steps from it, and training ends
    # on the last evaluated iterate: two iterations leave the first step
    m.train(torch.tensor(u), y, iters=2, lr=1e-3)
    th1, _ = m.get_params()
    mask = S.d_mask(4, NU, NY) > 0
    big = mask & (np.abs(g) > 1e-3 * np.abs(g).max())
    np.testing.assert_allclose(th1[big] - th32[big], -1e-3 * np.sign(g[big]), rtol=1e-3, atol=1e-7)
    m.set_params(th32, sc)
    hist = m.train(torch.tensor(u), y, iters=300, lr=3e-3).cpu().numpy()
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.5 * hist[0]
    th, _ = m.get_params()
    assert np.all(th[~mask] == 0)
    m.close()


def test_lbfgs_never_raises_the_loss_and_refines_adam():
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    teacher = _theta(4, 21, m1=0.1)[1]
    u, _ = _data(12, 80, 22, sc)
    mt = VelocityModel(nx=4)
    mt.set_params(teacher, sc)
    y, _ = mt.predict(torch.tensor(u), Ts=0.05)
    mt.close()
    m = VelocityModel(nx=4, sigma2=1e-6)
    m.set_params(_theta(4, 23, m1=0.05)[1], sc)
    m.train(torch.tensor(u), y, iters=100, lr=3e-3)
    l0 = float(m.loss_grad(torch.tensor(u), y, grad=False)[0].item())
    hist = m.lbfgs(torch.tensor(u), y, iters=40)
    l1 = float(m.loss_grad(torch.tensor(u), y, grad=False)[0].item())
    assert np.all(np.diff(hist) <= 0) and hist[0] <= l0 and l1 == pytest.approx(hist[-1], rel=1e-12)
    assert l1 < 0.9 * l0
    th, _ = m.get_params()
    assert np.all(th[S.d_mask(4, NU, NY) == 0] == 0)
    m.close()


def test_least_squares_start_matches_oracle():
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    teacher = _theta(4, 31, m1=0.1)[1]
    u, _ = _data(10, 150, 32, sc)
    mt = VelocityModel(nx=4)
    mt.set_params(teacher, sc)
    y, _ = mt.predict(torch.tensor(u), Ts=0.05)
    mt.close()
    yn = y.cpu().numpy()
    m = VelocityModel(nx=4)
    m.set_params(None, sc)
    m.init_ls(torch.tensor(u), y)
    th, _ = m.get_params()
    ref = S.ls_start([u[i].astype(np.float64) / sc[:3] for i in range(10)],
                     [yn[i].astype(np.float64) / sc[3:] for i in range(10)], 4)
    assert np.abs(th - ref).max() <= 1e-5 * np.abs(ref).max()
    m.close()


def test_scheduling_network_gains_over_the_lti_fit_when_the_system_is_scheduled():
    """On data of a strongly scheduled teacher, the LPV fit started on the best
    LTI fit (M_1 = 0, random network, then L-BFGS on all of theta) ends well
    below the LTI loss: what the trained network adds over the model without it."""
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel, initial_theta
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    teacher = _theta(4, 41, m1=0.3)[1]
    u, _ = _data(16, 120, 42, sc)
    mt = VelocityModel(nx=4)
    mt.set_params(teacher, sc)
    y, _ = mt.predict(torch.tensor(u), Ts=0.05)
    mt.close()
    ut = torch.tensor(u)
    m = VelocityModel(nx=4, sigma2=1e-6)
    m.normalize(ut, y)
    _, s = m.get_params()
    m.init_ls(ut, y)
    m.train(ut, y, iters=300, lr=1e-3, stage=m.LTI)
    m.lbfgs(ut, y, iters=100, stage=m.LTI)
    l_lti = float(m.loss_grad(ut, y, grad=False)[0].item())
    th_lti, _ = m.get_params()
    best = np.inf
    for r in range(3):
        m.set_params(initial_theta(4, seed=50 + r, base=th_lti, m1_std=0.0), s)
        l0 = float(m.loss_grad(ut, y, grad=False)[0].item())
        assert l0 == pytest.approx(l_lti, rel=1e-3)  # the restart starts on the LTI fit (plus the l2 term of the network)
        m.lbfgs(ut, y, iters=300)
        best = min(best, float(m.loss_grad(ut, y, grad=False)[0].item()))
    assert best < 0.8 * l_lti, (best, l_lti)
    m.close()


@pytest.mark.parametrize("nx,n_traj,T", [(8, 70, 25), (6, 65, 1), (4, 1, 3)])
def test_gradient_parity_at_edge_sizes(nx, n_traj, T):
    """The largest state (n_x = 8: 80 KB of per-thread accumulators, above the
    default shared-memory limit), more trajectories than one block holds (a
    ragged second block), a single sample, a single trajectory."""
    torch = need_gpu()
    from paper_2604_12505_gb300.slpv import VelocityModel
    sc = np.array([20.0, 20.0, 2.0, 0.1, 0.1, 0.05], dtype=np.float32)
    th64, th32 = _theta(nx, 60 + nx, m1=0.1)
    u, y = _data(n_traj, T, 61, sc)
    U = [u[i].astype(np.float64) / sc[:3] for i in range(n_traj)]
    Y = [y[i].astype(np.float64) / sc[3:] for i in range(n_traj)]
    ref_l = S.loss(th64, U, Y, nx, 1e-4)
    ref_g = S.loss_grad(th64, U, Y, nx, 1e-4, S.d_mask(nx, NU, NY))
    m = VelocityModel(nx=nx, sigma2=1e-4)
    m.set_params(th32, sc)
    loss, g = m.loss_grad(torch.tensor(u), torch.tensor(y))
    assert abs(float(loss.item()) - ref_l) <= 1e-4 * ref_l
    assert np.abs(g.cpu().numpy() - ref_g).max() <= 1e-3 * np.abs(ref_g).max()
    m.close()

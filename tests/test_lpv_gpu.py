"""GPU parity of the LPV surrogate kernels against the FP64 oracle (oracle/lpv.py).

Tolerances: the least-squares regression is FP64 on both sides (1e-8
relative); the start it gives is stored in FP32 (1e-5).
The recurrence, its adjoint and the closed loop run on tensor cores with
operands split into two BF16 halves (about 16 significant bits each, FP32
accumulation) and an FP32 rigid body: 1e-3 of the largest entry, norm-wise.
"""
import numpy as np
import pytest

from oracle import lpv as L
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
NX, NU, NY, NP = 12, 3, 4, 2


def _stable_W(rng, n_p=NP, scale=0.3):
    W = np.zeros((NX + NY, (1 + n_p) * (NX + NU)))
    for i in range(1 + n_p):
        A = rng.normal(size=(NX, NX))
        A *= (0.6 if i == 0 else 0.15) / np.linalg.norm(A, 2)  # ||A(p)||_2 <= 0.9 for |p_i| <= 1
        blk = slice(i * (NX + NU), (i + 1) * (NX + NU))
        W[:NX, blk] = np.concatenate([A, scale * rng.normal(size=(NX, NU))], axis=1)
        W[NX:, blk][:, :NX] = scale * rng.normal(size=(NY, NX))
    return W


def _data(rng, n, T, n_p=NP):
    from paper_2604_12505_gb300 import workloads as W
    u = np.stack([W.piecewise_profile(T, 0.05, seed=int(rng.integers(1 << 30)), hold=(0.1, 0.6), tau_amp=1.0,
                                      f_amp=1.0) for _ in range(n)])
    p = np.zeros((n, T, n_p))
    if n_p > 0:
        p[:, :, 0] = rng.uniform(-1, 1, size=(n, 1))
    if n_p > 1:
        p[:, :, 1] = np.sin(np.linspace(0, 6, T))[None] * rng.uniform(-1, 1, size=(n, 1))
    return u, p


def _unit_scales(n_p=NP):
    return np.concatenate([np.ones(NU), np.ones(NY), np.zeros(n_p), np.ones(n_p), np.full(n_p, -np.inf),
                           np.full(n_p, np.inf)]).astype(np.float32)


def _model(n_p=NP, **kw):
    from paper_2604_12505_gb300.lpv import Model
    return Model(dict(n_p=n_p, **kw))


def test_least_squares_start_matches_oracle():
    need_gpu()
    rng = np.random.default_rng(0)
    A = [0.3 * rng.normal(size=(NY, NY)) / (i + 1) for i in range(3)]
    B = [rng.normal(size=(NY, NU)) for _ in range(3)]
    u, _ = _data(rng, 21, 160)
    y = np.zeros((21, 160, NY))
    for b in range(21):
        for k in range(160):
            for i in range(1, 4):
                if k - i >= 0:
                    y[b, k] += A[i - 1] @ y[b, k - i] + B[i - 1] @ u[b, k - i]
    y += 0.01 * rng.normal(size=y.shape)
    # both sides get the same (FP32) data
    u = u.astype(np.float32).astype(np.float64)
    y = y.astype(np.float32).astype(np.float64)
    m = _model()
    m.set_params(scales=_unit_scales())
    theta = m.init_ls(u, y)
    Ao, Bo = L.arx_ls(list(u), list(y), 3, 3)
    th_o = np.concatenate([a.T for a in Ao] + [b.T for b in Bo], axis=0)
    np.testing.assert_allclose(theta, th_o, rtol=1e-8, atol=1e-10)
    W, _ = m.get_params()
    Wo = L.ls_start(list(u), list(y), 3, 0.999, NP).reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2)
    np.testing.assert_allclose(W, Wo, rtol=1e-5, atol=1e-6 * np.abs(Wo).max())
    # rho_max = 0 keeps the observer-canonical form of the plain fit
    m0 = _model(rho_max=0.0)
    m0.set_params(scales=_unit_scales())
    m0.init_ls(u, y)
    Wc = L.ss_to_W(*L.arx_to_ss(Ao, Bo), n_p=NP).reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2)
    np.testing.assert_allclose(m0.get_params()[0], Wc, rtol=1e-6, atol=1e-7)


def test_unstable_least_squares_start_is_scaled_like_the_oracle():
    need_gpu()
    rng = np.random.default_rng(10)
    # an ARX system with a root near 1.04: the estimate is unstable
    A = [np.diag([1.04, 0.5, 0.3, -0.2]) + 0.02 * rng.normal(size=(NY, NY)), 0.05 * rng.normal(size=(NY, NY)),
         0.02 * rng.normal(size=(NY, NY))]
    B = [rng.normal(size=(NY, NU)) for _ in range(3)]
    u, _ = _data(rng, 12, 60)
    y = np.zeros((12, 60, NY))
    for b in range(12):
        for k in range(60):
            for i in range(1, 4):
                if k - i >= 0:
                    y[b, k] += A[i - 1] @ y[b, k - i] + B[i - 1] @ u[b, k - i]
    y += 0.01 * rng.normal(size=y.shape)
    u = u.astype(np.float32).astype(np.float64)
    y = y.astype(np.float32).astype(np.float64)
    m = _model(rho_max=0.97)
    m.set_params(scales=_unit_scales())
    m.init_ls(u, y)
    Ao, Bo = L.arx_ls(list(u), list(y), 3, 3)
    assert L.stabilize(Ao, Bo, 0.97)[2] > 1.0
    Wo = L.ls_start(list(u), list(y), 3, 0.97, NP).reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2)
    W, _ = m.get_params()
    np.testing.assert_allclose(W, Wo, rtol=1e-5, atol=1e-6 * np.abs(Wo).max())
    A0 = W[0, :NX, :NX].astype(np.float64)
    assert np.abs(np.linalg.eigvals(A0)).max() == pytest.approx(0.97, rel=1e-5)
    # balanced: both Gramians equal and diagonal
    B0, C0 = W[0, :NX, NX:].astype(np.float64), W[0, NX:, :NX].astype(np.float64)
    P = np.zeros((NX, NX))
    Q = np.zeros((NX, NX))
    Ak = np.eye(NX)
    for _ in range(3000):
        P += Ak @ B0 @ B0.T @ Ak.T
        Q += Ak.T @ C0.T @ C0 @ Ak
        Ak = Ak @ A0
    np.testing.assert_allclose(P, Q, atol=1e-4 * np.abs(P).max())
    np.testing.assert_allclose(P, np.diag(np.diag(P)), atol=1e-4 * np.abs(P).max())


def test_normalisation_statistics():
    need_gpu()
    rng = np.random.default_rng(1)
    u, p = _data(rng, 19, 50)
    y = rng.normal(size=(19, 50, NY)) * np.array([1.0, 3.0, 0.2, 7.0])
    m = _model()
    m.normalize(u, y, p)
    _, s = m.get_params()
    np.testing.assert_allclose(s[:NU], np.sqrt((u ** 2).mean(axis=(0, 1))), rtol=1e-5)
    np.testing.assert_allclose(s[NU:NU + NY], np.sqrt((y ** 2).mean(axis=(0, 1))), rtol=1e-5)
    np.testing.assert_allclose(s[NU + NY:NU + NY + NP], p.mean(axis=(0, 1)), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(s[NU + NY + NP:NU + NY + 2 * NP], p.std(axis=(0, 1)), rtol=1e-4)
    p32 = p.astype(np.float32)
    np.testing.assert_array_equal(s[NU + NY + 2 * NP:NU + NY + 3 * NP], p32.min(axis=(0, 1)))
    np.testing.assert_array_equal(s[NU + NY + 3 * NP:], p32.max(axis=(0, 1)))


@pytest.mark.parametrize("n_traj,T", [(37, 40), (16, 7)])
def test_loss_and_bptt_gradient_match_oracle(n_traj, T):
    need_gpu()
    rng = np.random.default_rng(2)
    Wt = _stable_W(rng)
    u, p = _data(rng, n_traj, T)
    y = rng.normal(size=(n_traj, T, NY))
    m = _model(sigma2=1e-2)
    m.set_params(Wt.reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2), _unit_scales())
    W32 = m.get_params()[0].transpose(1, 0, 2).reshape(NX + NY, -1).astype(np.float64)
    loss, g = m.loss_grad(u, y, p)
    mask = L.d_mask(NX, NU, NY, NP)
    lo = L.loss(W32, list(u), list(y), list(p), NX, 1e-2)
    go = L.loss_grad(W32, list(u), list(y), list(p), NX, 1e-2, mask=mask)
    assert loss == pytest.approx(lo, rel=1e-4)
    g = g.transpose(1, 0, 2).reshape(NX + NY, -1)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    assert np.all(g[mask == 0] == 0)


def test_free_run_prediction_matches_oracle():
    need_gpu()
    rng = np.random.default_rng(3)
    Wt = _stable_W(rng)
    u, p = _data(rng, 33, 300)
    scales = np.concatenate([[2.0, 3.0, 0.5], [10.0, 20.0, 1.5, 0.1], [0.1, -0.2], [0.5, 2.0],
                             [-np.inf, -np.inf], [np.inf, np.inf]]).astype(np.float32)
    m = _model()
    m.set_params(Wt.reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2), scales)
    W32 = m.get_params()[0].transpose(1, 0, 2).reshape(NX + NY, -1).astype(np.float64)
    yg = m.predict(u, p).cpu().numpy()
    for b in range(33):
        pn = (p[b] - scales[7:9]) / scales[9:11]
        yo, _ = L.simulate(W32, u[b] / scales[:3], pn, NX)
        yo = yo * scales[3:7]
        assert np.abs(yg[b] - yo).max() <= 1e-3 * np.abs(yo).max()


def test_closed_loop_matches_oracle():
    need_gpu()
    rng = np.random.default_rng(4)
    Wt = _stable_W(rng, scale=0.05)
    B, T = 37, 200
    # the angular-rate range is narrower than the runs reach: the clamp is exercised
    scales = np.array([20.0, 20.0, 2.0, 30.0, 30.0, 3.0, 0.05, 0.5, 0.0, 0.2, 0.05, 0.2, -0.01, 0.8, 0.01],
                      dtype=np.float32)
    m = _model()
    m.set_params(Wt.reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2), scales)
    W32 = m.get_params()[0].transpose(1, 0, 2).reshape(NX + NY, -1).astype(np.float64)
    F = rng.uniform(-20, 20, size=(B, T, 2))
    tau = rng.uniform(-2, 2, size=(B, T))
    ref = np.repeat(rng.uniform(-0.1, 0.1, size=(B, T // 20)), 20, axis=1)
    fill = rng.uniform(0.2, 0.8, size=B)
    body = dict(m=500.0, J=50.0, Ts=0.005, n_sub=10, ctrl_omega=0.2 * np.pi, ctrl_xi=0.7)
    out = m.simulate(F, tau, ref, fill, body).cpu().numpy()
    clamped = 0
    sc = dict(u=scales[:3].astype(np.float64), y=scales[3:7].astype(np.float64),
              p_mean=scales[7:9].astype(np.float64), p_scale=scales[9:11].astype(np.float64))
    for b in range(B):
        o = L.closed_loop(W32, NX, sc, body, fill[b], F[b], tau[b], ref[b], body["Ts"], body["n_sub"],
                          dict(omega=body["ctrl_omega"], xi=body["ctrl_xi"]),
                          p_range=(scales[11:13].astype(np.float64), scales[13:15].astype(np.float64)))
        clamped += np.abs(o[:, 5]).max() > 0.01
        for cols in ([0, 1], [2], [3, 4], [5]):
            den = np.linalg.norm(o[:, cols], axis=1).max()
            assert np.linalg.norm(out[b][:, cols] - o[:, cols], axis=1).max() <= 1e-3 * den
    assert clamped > 0


def test_training_reduces_loss_and_scheduling_gains_over_lti():
    # Data from an LPV system whose dynamics depend on the scheduling: the
    # affine LPV model recovers it, a model without scheduling cannot.
    torch = need_gpu()
    rng = np.random.default_rng(5)
    Wt = _stable_W(rng)
    for i in (1, 2):  # strong scheduling of the input and output maps
        blk = slice(i * (NX + NU), (i + 1) * (NX + NU))
        Wt[:NX, blk][:, NX:] *= 4.0
        Wt[NX:, blk][:, :NX] *= 4.0
    u, p = _data(rng, 160, 120)
    y = np.stack([L.simulate(Wt, u[b], p[b], NX)[0] for b in range(160)])
    tr, te = slice(0, 128), slice(128, 160)
    from paper_2604_12505_gb300 import lpv
    res = {}
    for n_p in (0, 2):
        pp = p[:, :, :n_p]
        model, best = lpv.fit(u[tr], y[tr], pp[tr], dict(n_p=n_p, adam_iters=400, restarts=2, lr=3e-3, sigma2=1e-6))
        yh = model.predict(u[te], pp[te]).cpu().numpy()
        res[n_p] = np.mean([1 - L.bfr(y[b], yh[b - 128]) / 100 for b in range(128, 160)])
        # Adam from the least-squares start lowers the training loss
        m = lpv.Model(dict(n_p=n_p, lr=3e-3, sigma2=1e-6))
        m.normalize(u[tr], y[tr], pp[tr])
        m.init_ls(u[tr], y[tr])
        hist = m.train(u[tr], y[tr], pp[tr], 100)
        assert np.all(np.isfinite(hist)) and hist[-1] < hist[0], hist[[0, -1]]
    assert res[2] < 0.5 * res[0], res


def test_non_finite_steps_are_rejected_and_retried_smaller():
    # a step size of 3 throws the model far outside the stable region: the
    # free run overflows, the step is rejected and retried at half the size
    need_gpu()
    rng = np.random.default_rng(6)
    Wt = _stable_W(rng)
    u, p = _data(rng, 16, 400)
    y = np.stack([L.simulate(Wt, u[b], p[b], NX)[0] for b in range(16)])
    m = _model(lr=3.0)
    m.set_params(Wt.reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2), _unit_scales())
    hist = m.train(u, y, p, 40)
    assert np.isfinite(hist[0])
    assert not np.all(np.isfinite(hist)), "the test needs at least one overflowing step"
    assert np.isfinite(hist[-1])
    W, _ = m.get_params()
    assert np.all(np.isfinite(W))


def test_lbfgs_descends_monotonically_and_outpaces_adam_near_a_teacher():
    need_gpu()
    rng = np.random.default_rng(7)
    Wt = _stable_W(rng)
    u, p = _data(rng, 64, 80)
    y = np.stack([L.simulate(Wt, u[b], p[b], NX)[0] for b in range(64)])
    mask = L.d_mask(NX, NU, NY, NP)
    W0 = Wt + 0.02 * rng.normal(size=Wt.shape) * mask
    runs = {}
    for name in ("lbfgs", "adam"):
        m = _model(sigma2=0.0, lr=1e-3)
        m.set_params(W0.reshape(NX + NY, 1 + NP, NX + NU).transpose(1, 0, 2), _unit_scales())
        l0, _ = m.loss_grad(u, y, p)
        hist = m.lbfgs(u, y, p, 40) if name == "lbfgs" else m.train(u, y, p, 40)
        runs[name] = (l0, hist, m.get_params()[0])
    l0, h, Wl = runs["lbfgs"]
    assert np.all(np.diff(h) <= 0.0), h          # Armijo: accepted losses never increase
    assert h[-1] < 1e-2 * l0, (l0, h[-1])
    assert h[-1] < 0.25 * runs["adam"][1][-1], (h[-1], runs["adam"][1][-1])
    Wl = Wl.transpose(1, 0, 2).reshape(NX + NY, -1)
    assert np.all(Wl[mask == 0] == 0.0)


def test_fit_with_lbfgs_ends_no_worse_than_adam_alone():
    need_gpu()
    from paper_2604_12505_gb300 import lpv
    rng = np.random.default_rng(8)
    Wt = _stable_W(rng)
    u, p = _data(rng, 48, 60)
    y = np.stack([L.simulate(Wt, u[b], p[b], NX)[0] for b in range(48)])
    cfg = dict(adam_iters=100, restarts=2, lr=3e-3, sigma2=1e-6)
    _, best_adam = lpv.fit(u, y, p, cfg)
    _, best_both = lpv.fit(u, y, p, dict(cfg, lbfgs_iters=50))
    assert np.isfinite(best_both) and best_both <= best_adam


def test_concurrent_restarts_equal_the_restarts_run_alone():
    # The restarts of lpv_fit run concurrently (a model, a stream and a host
    # thread each).  Restart r draws its M_i from the seed + 1000003 r, so a
    # fit with one restart and that seed is restart r alone: the best loss
    # of the concurrent fit is the least of those, bit for bit, and its
    # weights are that restart's weights.
    need_gpu()
    from paper_2604_12505_gb300 import lpv
    rng = np.random.default_rng(9)
    Wt = _stable_W(rng)
    u, p = _data(rng, 40, 50)
    y = np.stack([L.simulate(Wt, u[b], p[b], NX)[0] for b in range(40)])
    cfg = dict(adam_iters=60, lbfgs_iters=20, lr=3e-3, sigma2=1e-6, init_scale=0.05, seed=11)
    model, best = lpv.fit(u, y, p, dict(cfg, restarts=4))
    alone = [lpv.fit(u, y, p, dict(cfg, restarts=1, seed=11 + 1000003 * r)) for r in range(4)]
    losses = [b for _, b in alone]
    assert len(set(losses)) > 1
    r = int(np.argmin(losses))
    assert best == losses[r]
    np.testing.assert_array_equal(model.get_params()[0], alone[r][0].get_params()[0])

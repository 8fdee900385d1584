"""Pins of the FP64 LPV oracle (Section 4) against closed forms, exact
recovery, finite differences and the SPH oracle's rigid body."""
import numpy as np
import pytest

from oracle import lpv as L


def test_scalar_impulse_response_closed_form():
    a, b, c = 0.8, 1.5, -0.7
    W = np.array([[a, b], [c, 0.0]])           # nx = nu = ny = 1, no scheduling
    T = 12
    u = np.zeros((T, 1))
    u[0] = 1.0
    y, x = L.simulate(W, u, np.zeros((T, 0)), nx=1)
    expect = np.array([0.0] + [c * a ** (k - 1) * b for k in range(1, T)])
    np.testing.assert_allclose(y[:, 0], expect, rtol=1e-14, atol=1e-15)


def test_affine_scheduling_with_constant_p_is_lti():
    rng = np.random.default_rng(0)
    nx, nu, ny, n_p = 3, 2, 2, 2
    W = 0.3 * rng.normal(size=(nx + ny, (1 + n_p) * (nx + nu)))
    p = np.array([0.4, -1.3])
    M = W[:, :nx + nu] + p[0] * W[:, nx + nu:2 * (nx + nu)] + p[1] * W[:, 2 * (nx + nu):]
    u = rng.normal(size=(20, nu))
    y1, _ = L.simulate(W, u, np.tile(p, (20, 1)), nx)
    y2, _ = L.simulate(M, u, np.zeros((20, 0)), nx)
    np.testing.assert_allclose(y1, y2, rtol=1e-12, atol=1e-14)


def _true_arx(rng, ny, nu, n):
    A = [0.25 * rng.normal(size=(ny, ny)) / (i + 1) for i in range(n)]
    B = [rng.normal(size=(ny, nu)) for _ in range(n)]
    return A, B


def _arx_sim(A, B, u):
    T, ny = u.shape[0], A[0].shape[0]
    y = np.zeros((T, ny))
    for k in range(T):
        for i in range(1, len(A) + 1):
            if k - i >= 0:
                y[k] += A[i - 1] @ y[k - i] + B[i - 1] @ u[k - i]
    return y


def test_arx_least_squares_recovers_a_noise_free_system():
    rng = np.random.default_rng(1)
    A, B = _true_arx(rng, 4, 3, 3)
    U = [rng.normal(size=(300, 3)) for _ in range(3)]
    Y = [_arx_sim(A, B, u) for u in U]
    Ah, Bh = L.arx_ls(U, Y, 3, 3)
    for i in range(3):
        np.testing.assert_allclose(Ah[i], A[i], atol=1e-9)
        np.testing.assert_allclose(Bh[i], B[i], atol=1e-9)


def test_observer_canonical_form_reproduces_the_arx_recursion():
    rng = np.random.default_rng(2)
    A, B = _true_arx(rng, 4, 3, 3)
    u = rng.normal(size=(60, 3))
    As, Bs, Cs = L.arx_to_ss(A, B)
    assert As.shape == (12, 12)
    W = L.ss_to_W(As, Bs, Cs, n_p=0)
    y_ss, _ = L.simulate(W, u, np.zeros((60, 0)), nx=12)
    np.testing.assert_allclose(y_ss, _arx_sim(A, B, u), rtol=1e-12, atol=1e-12)


def test_stabilize_scales_known_roots():
    # scalar ARX(2) with roots 1.1 and 0.5: a1 = r1 + r2, a2 = -r1 r2
    r1, r2, rho_max = 1.1, 0.5, 0.99
    A = [np.array([[r1 + r2]]), np.array([[-r1 * r2]])]
    B = [np.array([[1.0]]), np.array([[0.3]])]
    As, Bs, rho = L.stabilize(A, B, rho_max)
    lam = rho_max / r1
    assert rho == pytest.approx(r1, rel=1e-13)
    assert As[0][0, 0] == pytest.approx(lam * (r1 + r2), rel=1e-13)
    assert As[1][0, 0] == pytest.approx(-lam * lam * r1 * r2, rel=1e-13)
    assert Bs[0][0, 0] == pytest.approx(lam, rel=1e-13)
    assert Bs[1][0, 0] == pytest.approx(0.3 * lam * lam, rel=1e-13)
    # a stable model is left alone
    A2, B2, rho2 = L.stabilize([np.array([[0.5]])], [np.array([[2.0]])], rho_max)
    assert rho2 == pytest.approx(0.5) and A2[0][0, 0] == 0.5 and B2[0][0, 0] == 2.0


def test_stabilize_discounts_the_impulse_response():
    rng = np.random.default_rng(3)
    A = [0.9 * rng.normal(size=(2, 2)) for _ in range(3)]
    B = [rng.normal(size=(2, 1)) for _ in range(3)]
    As, Bs, rho = L.stabilize(A, B, 0.95)
    assert rho > 0.95
    lam = 0.95 / rho
    T = 40
    u = np.zeros((T, 1))
    u[0] = 1.0
    h, hs = _arx_sim(A, B, u), _arx_sim(As, Bs, u)
    np.testing.assert_allclose(hs, h * lam ** np.arange(T)[:, None], rtol=1e-10, atol=1e-12 * np.abs(h).max())


def test_balance_first_order_closed_form():
    # P = b^2 / (1 - a^2), Q = c^2 / (1 - a^2): S = |b c| / (1 - a^2), |b'| = |c'| = sqrt(|b c|)
    a, b, c = 0.9, 3.0, -0.5
    Ab, Bb, Cb, S = L.balance(np.array([[a]]), np.array([[b]]), np.array([[c]]), reg=0.0)
    assert S[0] == pytest.approx(abs(b * c) / (1 - a * a), rel=1e-12)
    assert Ab[0, 0] == pytest.approx(a, rel=1e-14)
    assert Cb[0, 0] == pytest.approx(np.sqrt(abs(b * c)), rel=1e-12)
    assert Bb[0, 0] == pytest.approx(np.sign(b * c) * np.sqrt(abs(b * c)), rel=1e-12)


def test_balance_gramians_by_direct_sums_and_markov_parameters():
    rng = np.random.default_rng(4)
    A, B = _true_arx(rng, 2, 2, 3)
    As, Bs, Cs = L.arx_to_ss(A, B)
    assert np.abs(np.linalg.eigvals(As)).max() < 0.8
    Ab, Bb, Cb, S = L.balance(As, Bs, Cs, reg=0.0)
    # Gramians as the series sum_k A^k B B^T A^kT (and the dual), truncated where it has converged
    P = np.zeros_like(Ab)
    Q = np.zeros_like(Ab)
    Ak = np.eye(len(Ab))
    for _ in range(400):
        P += Ak @ Bb @ Bb.T @ Ak.T
        Q += Ak.T @ Cb.T @ Cb @ Ak
        Ak = Ak @ Ab
    np.testing.assert_allclose(P, np.diag(S), atol=1e-9 * S.max())
    np.testing.assert_allclose(Q, np.diag(S), atol=1e-9 * S.max())
    assert np.all(np.diff(S) <= 0)
    M1, M2 = Cs @ Bs, Cb @ Bb
    A1, A2 = np.eye(len(As)), np.eye(len(Ab))
    for _ in range(30):
        np.testing.assert_allclose(M2, M1, atol=1e-10 * np.abs(Cs @ Bs).max())
        A1, A2 = A1 @ As, A2 @ Ab
        M1, M2 = Cs @ A1 @ Bs, Cb @ A2 @ Bb
    assert np.all(Cb[np.argmax(np.abs(Cb), axis=0), np.arange(len(Ab))] > 0)


def test_bptt_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    nx, nu, ny, n_p = 3, 2, 2, 2
    mask = L.d_mask(nx, nu, ny, n_p)
    W = 0.3 * rng.normal(size=mask.shape) * mask
    U = [rng.normal(size=(15, nu)) for _ in range(2)]
    P = [rng.uniform(-1, 1, size=(15, n_p)) for _ in range(2)]
    Y = [rng.normal(size=(15, ny)) for _ in range(2)]
    G = L.loss_grad(W, U, Y, P, nx, sigma2=1e-2, mask=mask)
    e = 1e-6
    for idx in [(0, 0), (1, 4), (2, 7), (3, 1), (4, 12), (0, 14), (4, 3)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += e
        Wm[idx] -= e
        fd = (L.loss(Wp, U, Y, P, nx, 1e-2) - L.loss(Wm, U, Y, P, nx, 1e-2)) / (2 * e)
        assert G[idx] == pytest.approx(fd * mask[idx], rel=1e-6, abs=1e-9)
    assert np.all(G[mask == 0] == 0)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = L.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-12)


def test_closed_loop_without_sloshing_matches_the_sph_oracle_rigid_body(orc):
    # a zero surrogate leaves the rigid body with PD control, which the SPH
    # oracle integrates with no fluid particles (independent code)
    from paper_2604_12505_gb300 import workloads as Wk
    Ts, n_sub, T = 0.05, 10, 80
    cfg = dict(Wk.SMALL, dt=Ts / n_sub, outer_every=n_sub)
    p = orc.params(**cfg)
    rng = np.random.default_rng(4)
    F = rng.uniform(-20, 20, size=(T, 2))
    tau = rng.uniform(-2, 2, size=T)
    ref = np.repeat(rng.uniform(-0.2, 0.2, size=T // 20), 20)
    u_inner = np.repeat(np.concatenate([F, tau[:, None]], axis=1), n_sub, axis=0)
    _, _, _, ysph, _ = orc.run(p, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(6), T * n_sub,
                               u=u_inner, theta_ref=ref, use_ctrl=True)
    W = np.zeros((16, 45))
    scales = dict(u=np.ones(3), y=np.ones(4), p_mean=np.zeros(2), p_scale=np.ones(2))
    out = L.closed_loop(W, 12, scales, dict(m=p.m_body, J=p.J_body), 0.5, F, tau, ref, Ts, n_sub,
                        dict(omega=p.ctrl_omega, xi=p.ctrl_xi))
    np.testing.assert_allclose(out, ysph[:, :6], rtol=1e-12, atol=1e-12)


def test_bfr_limits():
    rng = np.random.default_rng(5)
    y = rng.normal(size=(50, 3))
    np.testing.assert_allclose(L.bfr(y, y), 100.0)
    np.testing.assert_allclose(L.bfr(y, np.tile(y.mean(0), (50, 1))), 0.0, atol=1e-12)

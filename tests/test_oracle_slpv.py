"""Pins of the FP64 oracle of the self-scheduled LPV surrogate (Section 4,
Section 5.3.2) against closed forms and finite differences."""
import numpy as np
import pytest

from oracle import slpv as S

NX, NU, NY = 4, 3, 3


def _random_theta(seed, scale_m1=0.05):
    rng = np.random.default_rng(seed)
    P = {
        "M0": rng.normal(0, 0.3, (NX + NY, NX + NU)),
        "M1": rng.normal(0, scale_m1, (NX + NY, NX + NU)),
        "W1": rng.normal(0, 0.5, (4, NX + NU)),
        "b1": rng.normal(0, 0.1, 4),
        "W2": rng.normal(0, 0.5, (4, 4)),
        "b2": rng.normal(0, 0.1, 4),
        "w3": rng.normal(0, 0.5, 4),
        "b3": rng.normal(0, 0.1, 1),
    }
    P["M0"][:NX, :NX] *= 0.5  # a contracting A_0
    return S.pack(P) * S.d_mask(NX, NU, NY)


def test_parameter_count_and_layout():
    n = sum(S.sizes(NX, NU, NY))
    # two (nx+ny) x (nx+nu) matrices and a 7-4-4-1 network: 2*49 + 32 + 20 + 5
    assert n == 2 * 49 + (4 * 7 + 4) + (16 + 4) + (4 + 1) == 155
    assert int(S.d_mask(NX, NU, NY).sum()) == n - 2 * NY * NU  # the D blocks are fixed at zero
    th = _random_theta(0)
    np.testing.assert_array_equal(S.pack(S.unpack(th, NX, NU, NY)), th)


def test_without_scheduling_matrix_the_model_is_lti():
    """M_1 = 0: y_k = sum_j C A^(k-1-j) B u_j (impulse-response convolution)."""
    th = _random_theta(1)
    P = S.unpack(th, NX, NU, NY)
    P["M1"][:] = 0.0
    th = S.pack(P)
    A, B, C = P["M0"][:NX, :NX], P["M0"][:NX, NX:], P["M0"][NX:, :NX]
    u = np.random.default_rng(2).normal(size=(25, NU))
    y, _, _ = S.simulate(th, u, NX, NY)
    ref = np.zeros_like(y)
    for k in range(25):
        for j in range(k):
            ref[k] += C @ np.linalg.matrix_power(A, k - 1 - j) @ B @ u[j]
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


def test_constant_network_output_gives_the_frozen_lti_model():
    """W1 = W2 = 0: eta is the constant w3 . tanh(b2) + b3 for every z, so the
    model is the LTI system M_0 + p M_1 with that constant p."""
    th = _random_theta(3, scale_m1=0.3)
    P = S.unpack(th, NX, NU, NY)
    P["W1"][:] = 0.0
    P["W2"][:] = 0.0
    th = S.pack(P)
    pbar = float(P["w3"] @ np.tanh(P["b2"]) + P["b3"][0])
    M = P["M0"] + pbar * P["M1"]
    A, B, C = M[:NX, :NX], M[:NX, NX:], M[NX:, :NX]
    u = np.random.default_rng(4).normal(size=(20, NU))
    y, _, p = S.simulate(th, u, NX, NY)
    np.testing.assert_allclose(p, pbar, rtol=0, atol=1e-15)
    ref = np.zeros_like(y)
    for k in range(20):
        for j in range(k):
            ref[k] += C @ np.linalg.matrix_power(A, k - 1 - j) @ B @ u[j]
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


def test_scheduling_depends_on_state_and_input():
    th = _random_theta(5, scale_m1=0.3)
    u = np.random.default_rng(6).normal(size=(15, NU))
    _, _, p = S.simulate(th, u, NX, NY)
    assert np.ptp(p) > 1e-3


def test_bptt_gradient_matches_central_differences():
    th = _random_theta(7, scale_m1=0.2)
    rng = np.random.default_rng(8)
    U = [rng.normal(size=(12, NU)) for _ in range(2)]
    Y = [rng.normal(size=(12, NY)) for _ in range(2)]
    mask = S.d_mask(NX, NU, NY)
    g = S.loss_grad(th, U, Y, NX, 1e-3, mask)
    eps = 1e-6
    fd = np.zeros_like(th)
    for i in np.flatnonzero(mask):
        e = np.zeros_like(th)
        e[i] = eps
        fd[i] = (S.loss(th + e, U, Y, NX, 1e-3) - S.loss(th - e, U, Y, NX, 1e-3)) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())
    assert np.all(g[mask == 0] == 0)


def test_augmentation_integrates_the_velocity_output():
    """e_k = Ts * sum_{j<k} y_j: for the LTI model C = I, A = I, B = Ts I/m
    (a rigid body at the velocity level) a constant input gives the discrete
    double integrator e_k = Ts^2 u/m * k (k - 1) / 2."""
    P = S.unpack(np.zeros(sum(S.sizes(NX, NU, NY))), NX, NU, NY)
    Ts, m = 0.05, 2.0
    P["M0"][:3, :3] = np.eye(3)
    P["M0"][:3, NX:] = Ts / m * np.eye(3)
    P["M0"][NX:, :3] = np.eye(3)
    th = S.pack(P)
    u = np.tile([1.0, -2.0, 0.5], (30, 1))
    e, yh = S.augment(th, u, NX, NY, Ts)
    k = np.arange(30)[:, None]
    np.testing.assert_allclose(yh, Ts / m * k * u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(e, Ts * Ts / m * u * k * (k - 1) / 2, rtol=0, atol=1e-13)


def test_closed_loop_of_a_rigid_body_model_is_the_discrete_pd_loop():
    """A velocity-level rigid body (A = I, B = Ts/J on the torque channel,
    C = I) under Eq. 28 gives the linear recursion [theta, w]_{k+1} =
    Phi [theta, w]_k + Gamma theta_ref with Phi = [[1, Ts], [-Ts w^2,
    1 - 2 xi w Ts]] in the torque-normalised units, computed here by matrix
    powers."""
    J, wn, xi, Ts = 50.0, 0.2 * np.pi, 0.7, 0.05
    P = S.unpack(np.zeros(sum(S.sizes(NX, NU, NY))), NX, NU, NY)
    P["M0"][:3, :3] = np.eye(3)
    P["M0"][2, NX + 2] = Ts / J       # normalised input u / s_u with s_u = 1
    P["M0"][NX:, :3] = np.eye(3)
    th = S.pack(P)
    T = 400  # 20 s: twice the settling time of the 0.1 Hz, xi = 0.7 loop
    F = np.zeros((T, 2))
    tau = np.zeros(T)
    ref = np.full(T, 0.3)
    out = S.closed_loop(th, NX, dict(u=np.ones(3), y=np.ones(3)), F, tau, ref, Ts, dict(J=J, omega=wn, xi=xi))
    Phi = np.array([[1.0, Ts], [-Ts * wn * wn, 1.0 - 2.0 * xi * wn * Ts]])
    Gam = np.array([0.0, Ts * wn * wn])
    s = np.zeros(2)
    traj = []
    for k in range(T):
        traj.append(s.copy())
        s = Phi @ s + Gam * ref[k]
    traj = np.array(traj)
    np.testing.assert_allclose(out[:, 2], traj[:, 0], rtol=0, atol=1e-12)
    # thetadot sample of step k is C x_k with x_k the rate before the kick of step k
    np.testing.assert_allclose(out[:, 5], traj[:, 1], rtol=0, atol=1e-12)
    assert abs(out[-1, 2] - 0.3) < 1e-3  # the loop settles on the reference


def test_ls_start_recovers_a_first_order_system_exactly():
    """Noise-free data of y_{k+1} = A1 y_k + B1 u_k (y_0 = 0) give back A1 and
    B1, and the realised start reproduces the data in free run."""
    rng = np.random.default_rng(30)
    A1 = np.diag([0.99, 0.95, 0.9]) + 0.01 * rng.normal(size=(3, 3))
    B1 = rng.normal(0, 0.2, (3, 3))
    U, Y = [], []
    for _ in range(3):
        u = rng.normal(size=(40, NU))
        y = np.zeros((40, NY))
        for k in range(39):
            y[k + 1] = A1 @ y[k] + B1 @ u[k]
        U.append(u)
        Y.append(y)
    th = S.ls_start(U, Y, NX)
    P = S.unpack(th, NX, NU, NY)
    np.testing.assert_allclose(P["M0"][:3, :3], A1, atol=1e-10)
    np.testing.assert_allclose(P["M0"][:3, NX:], B1, atol=1e-10)
    assert np.all(P["M0"][3, :] == 0) and np.all(P["M1"] == 0)
    yh, _, _ = S.simulate(th, U[0], NX, NY)
    np.testing.assert_allclose(yh, Y[0], atol=1e-9)


def test_closed_loop_equals_the_free_run_under_the_inputs_it_applied():
    """With a network that ignores the input, the scheduling at the sample and
    at the step coincide, so the closed loop (scheduled, M_1 != 0) must equal
    the open-loop free run and augmentation driven by the inputs the PD law
    applied, rebuilt from the recorded angle and rate."""
    th = _random_theta(70, scale_m1=0.3)
    P = S.unpack(th, NX, NU, NY)
    P["W1"][:, NX:] = 0.0                       # eta depends on the state only
    th = S.pack(P)
    rng = np.random.default_rng(71)
    T, Ts = 60, 0.05
    su, sy = np.array([20.0, 20.0, 2.0]), np.array([0.1, 0.1, 0.05])
    F = rng.uniform(-20, 20, (T, 2))
    tau = rng.uniform(-2, 2, T)
    ref = np.full(T, 0.2)
    pd = dict(J=133.84, omega=0.2 * np.pi, xi=0.7)
    out = S.closed_loop(th, NX, dict(u=su, y=sy), F, tau, ref, Ts, pd)
    J, w, xi = pd["J"], pd["omega"], pd["xi"]
    tc = J * w * w * (ref - out[:, 2]) - 2.0 * xi * J * w * out[:, 5]
    u = np.column_stack([F, tau + tc]) / su
    e, yh = S.augment(th, u, NX, NY, Ts)
    np.testing.assert_allclose(out[:, 3:], yh * sy, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, :3], e * sy, rtol=0, atol=1e-12)


def test_scheduling_network_equals_an_independent_tanh_network():
    """eta is the two-hidden-layer tanh network of Section 5.3.2 on z = [x, u]:
    evaluated by torch.nn layers (Linear, Tanh, Linear, Tanh, Linear) loaded
    with the same weights, at the states and inputs of a free run."""
    torch = pytest.importorskip("torch")
    th = _random_theta(7, scale_m1=0.3)
    P = S.unpack(th, NX, NU, NY)
    net = torch.nn.Sequential(torch.nn.Linear(NX + NU, 4), torch.nn.Tanh(), torch.nn.Linear(4, 4), torch.nn.Tanh(),
                              torch.nn.Linear(4, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.tensor(P["W1"]))
        net[0].bias.copy_(torch.tensor(P["b1"]))
        net[2].weight.copy_(torch.tensor(P["W2"]))
        net[2].bias.copy_(torch.tensor(P["b2"]))
        net[4].weight.copy_(torch.tensor(P["w3"][None, :]))
        net[4].bias.copy_(torch.tensor(P["b3"]))
    u = np.random.default_rng(8).normal(size=(30, NU))
    _, xs, ps = S.simulate(th, u, NX, NY)
    z = np.concatenate([xs[:-1], u], axis=1)                 # z_k = [x_k; u_k]
    with torch.no_grad():
        ref = net(torch.tensor(z)).numpy()[:, 0]
    np.testing.assert_allclose(ps, ref, rtol=0, atol=1e-14)
    assert np.ptp(ps) > 0.1                                   # the network is not at a constant
    # a hand-worked case: one active neuron per layer
    Q = {k: np.zeros_like(v) for k, v in P.items()}
    Q["W1"][0, 1] = 2.0
    Q["b1"][0] = 0.5
    Q["W2"][0, 0] = -1.5
    Q["w3"][0] = 3.0
    Q["b3"][0] = 0.25
    z1 = np.zeros(NX + NU)
    z1[1] = 0.4
    p1, _, _ = S.eta(Q, z1)
    assert p1 == pytest.approx(3.0 * np.tanh(-1.5 * np.tanh(2.0 * 0.4 + 0.5)) + 0.25, abs=1e-15)

"""Pins of the SPH oracle (Section 3, Algorithm 1) against closed forms,
brute force, conservation laws and finite differences.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2604_12505_gb300 import workloads as W

SIG = 5.0 / (14.0 * math.pi)


def _p(orc, **kw):
    return orc.params(**dict(W.BASE, **kw))


# --------------------------------------------------------------------------
# tank construction
# --------------------------------------------------------------------------
def test_fill_chord_area(orc):
    R = 0.5
    for fill in (0.2, 0.5, 0.6, 0.8):
        c = orc.fill_chord(R, fill)
        area, _ = integrate.quad(lambda y: 2.0 * math.sqrt(max(R * R - y * y, 0.0)), -R, c, epsabs=1e-14)
        assert area == pytest.approx(fill * math.pi * R * R, rel=1e-12)
    assert orc.fill_chord(R, 0.5) == pytest.approx(0.0, abs=1e-15)


def test_tank_geometry(orc):
    p = _p(orc)
    x, gB = orc.tank(p)
    R, dx = p.R, p.dx
    # rings at R + (k + 1/2) dx with round(2 pi r_k / dx) equispaced ghosts
    radii = np.hypot(gB[:, 0], gB[:, 1])
    expect = [round(2 * math.pi * (R + (k + 0.5) * dx) / dx) for k in range(3)]
    assert gB.shape[0] == sum(expect) == 500
    off = 0
    for k, n in enumerate(expect):
        np.testing.assert_allclose(radii[off:off + n], R + (k + 0.5) * dx, rtol=1e-14)
        ang = np.unwrap(np.arctan2(gB[off:off + n, 1], gB[off:off + n, 0]))
        np.testing.assert_allclose(np.diff(ang), 2 * math.pi / n, rtol=1e-9)
        off += n
    # fluid on the half-offset lattice, inside R - dx/2 and below the chord
    assert np.all(np.hypot(x[:, 0], x[:, 1]) <= R - dx / 2 + 1e-15)
    assert np.all(x[:, 1] <= orc.fill_chord(R, 0.5) + 1e-15)
    frac = (x / dx - 0.5)
    np.testing.assert_allclose(frac, np.round(frac), atol=1e-9)
    # count close to the segment area over the cell area
    assert x.shape[0] == pytest.approx(0.5 * math.pi * R * R / dx**2, rel=0.05)


# --------------------------------------------------------------------------
# closed forms for a few particles
# --------------------------------------------------------------------------
def test_two_particle_density_and_forces(orc):
    p = _p(orc, dx=0.01, h_over_dx=1.3, alpha=0.3)
    h, m = orc.h_of(p), orc.mass_of(p)
    d = 0.7 * h
    x = np.array([[0.0, 0.0], [d * 0.6, d * 0.8]])
    v = np.array([[0.1, -0.2], [-0.3, 0.05]])
    body = np.array([10.0, 10.0, 0.0, 0.0, 0.0, 0.0])  # ghosts far away
    out = orc.evaluate(p, x, v, np.zeros((0, 2)), body)
    rho = m * (orc.w_cubic(0, h, SIG) + orc.w_cubic(d, h, SIG))  # Eq. 14 with the self term
    np.testing.assert_allclose(out["rho"], [rho, rho], rtol=1e-14)
    P = p.k * (rho - p.rho0)                                       # Eq. 11
    np.testing.assert_allclose(out["P"], [P, P], rtol=1e-13)
    r12 = x[0] - x[1]
    v12 = v[0] - v[1]
    gradW = orc.dw_cubic(d, h, SIG) / d * r12
    a1 = m * (-(2 * P / rho**2) + 2 * p.alpha * h / (2 * rho) * (v12 @ r12) / (d * d + p.eps * h * h)) * gradW
    np.testing.assert_allclose(out["acc"][0], a1, rtol=1e-12)
    np.testing.assert_allclose(out["acc"][1], -a1, rtol=1e-12)      # antisymmetry of Eqs. 10, 12
    np.testing.assert_allclose(out["fb"], 0.0, atol=0)


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_fluid_ghost_pair_closed_form(orc, sign):
    p = _p(orc, dx=0.01, ghost_pressure_sign=sign, beta=0.7)
    h, m = orc.h_of(p), orc.mass_of(p)
    gB = np.array([[0.2, 0.0]])
    body = np.array([0.01, -0.02, 0.3, 0.5, -0.4, 2.0])
    gw, gv, arm = orc.ghost_world(gB, body)
    d = 0.6 * h
    x = gw + np.array([[-d * 0.8, d * 0.6]])
    v = np.array([[-0.2, 0.3]])
    out = orc.evaluate(p, x, v, gB, body, u=(0.0, 0.0, 0.0))
    rho = m * (orc.w_cubic(0, h, SIG) + p.gamma1 * orc.w_cubic(d, h, SIG))
    P = p.k * (rho - p.rho0)
    r = x[0] - gw[0]
    gradWs = orc.dw_spiky(d, h) / d * r
    fp = sign * 2 * m * m * P / rho**2 * gradWs                         # Eq. 16
    vr = (v[0] - gv[0]) @ r
    fv = m * m * 2 * p.beta / (2 * rho) * min(vr, 0.0) / (d * d + p.eps * h * h) * gradWs  # Eq. 18
    f = fp + fv
    np.testing.assert_allclose(out["acc"][0], f / m, rtol=1e-12)
    np.testing.assert_allclose(out["fb"][:2], -f, rtol=1e-12)         # Eqs. 17, 19, 20
    np.testing.assert_allclose(out["fb"][2], -(arm[0, 0] * f[1] - arm[0, 1] * f[0]), rtol=1e-12)
    # with the default sign a compressed particle is pushed away from the wall
    if sign < 0 and P > 0:
        assert out["acc"][0] @ r > 0


def test_ghost_kinematics(orc):
    gB = np.array([[1.0, 0.0], [0.0, 2.0]])
    body = np.array([0.5, -1.0, math.pi / 2, 0.0, 0.0, 0.0])
    gw, _, _ = orc.ghost_world(gB, body)
    np.testing.assert_allclose(gw, [[0.5, 0.0], [-1.5, -1.0]], atol=1e-15)   # Eq. 21, R(pi/2)
    # velocity equals the time derivative of the position under the body motion
    body = np.array([0.1, 0.2, 0.7, 0.3, -0.6, 1.3])
    gw, gv, _ = orc.ghost_world(gB, body)
    e = 1e-6
    bp = body.copy(); bp[:3] += e * body[3:]
    bm = body.copy(); bm[:3] -= e * body[3:]
    fd = (orc.ghost_world(gB, bp)[0] - orc.ghost_world(gB, bm)[0]) / (2 * e)
    np.testing.assert_allclose(gv, fd, rtol=1e-8)


# --------------------------------------------------------------------------
# neighbour search, brute force vs bucket grid
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", [W.TINY, W.SMALL])
def test_bucket_grid_matches_brute_force(orc, cfg):
    p = orc.params(**cfg)
    x, gB = orc.tank(p)
    x = x + W.perturbation(x.shape, 0.2 * p.dx, seed=1)
    v = W.perturbation(x.shape, 0.3, seed=2)
    body = np.array([0.003, -0.002, 0.4, 0.1, -0.05, 0.7])
    a = orc.evaluate(p, x, v, gB, body, u=(1.0, 2.0, 3.0), brute=False)
    b = orc.evaluate(p, x, v, gB, body, u=(1.0, 2.0, 3.0), brute=True)
    for key in ("rho", "P", "acc", "drho", "fb", "body_acc"):
        scale = np.abs(b[key]).max()
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-13 * scale)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def test_closed_fluid_pair_forces_conserve_momentum(orc):
    # No ghosts: the symmetric forms of Eqs. 10 and 12 give zero net force and
    # zero net torque (central pair forces).
    p = orc.params(**W.TINY)
    x, _ = orc.tank(p)
    x = x + W.perturbation(x.shape, 0.25 * p.dx, seed=3)
    v = W.perturbation(x.shape, 0.5, seed=4)
    out = orc.evaluate(p, x, v, np.zeros((0, 2)), np.array([5.0, 5.0, 0, 0, 0, 0]))
    m = orc.mass_of(p)
    f = m * out["acc"]
    scale = np.abs(f).sum()
    assert abs(f[:, 0].sum()) < 1e-13 * scale
    assert abs(f[:, 1].sum()) < 1e-13 * scale
    torque = x[:, 0] * f[:, 1] - x[:, 1] * f[:, 0]
    assert abs(torque.sum()) < 1e-13 * np.abs(torque).sum()


def _momenta(orc, p, x, v, body):
    m = orc.mass_of(p)
    px = m * v[:, 0].sum() + p.m_body * body[3]
    py = m * v[:, 1].sum() + p.m_body * body[4]
    L = m * (x[:, 0] * v[:, 1] - x[:, 1] * v[:, 0]).sum() + p.m_body * (body[0] * body[4] - body[1] * body[3]) \
        + p.J_body * body[5]
    return np.array([px, py]), L


def test_symplectic_euler_conserves_momentum_of_fluid_and_body(orc):
    # Zero gravity, no input: kick-then-drift with central, antisymmetric pair
    # forces (fluid-fluid and fluid-ghost) conserves linear and angular
    # momentum of fluid plus body at every step (Section 3.4, Eq. 20).
    p = orc.params(**dict(W.TINY, dt=5e-5))
    x, gB = orc.tank(p)
    v = np.zeros_like(x)
    body = np.array([0.0, 0.0, 0.0, 0.02, -0.01, 0.5])
    p0, L0 = _momenta(orc, p, x, v, body)
    x1, v1, b1, _, _ = orc.run(p, x, v, gB, body, 2000, record=False)
    p1, L1 = _momenta(orc, p, x1, v1, b1)
    m = orc.mass_of(p)
    pscale = m * np.abs(v1).sum() + p.m_body * np.abs(b1[3:5]).sum()
    Lscale = m * np.abs(x1[:, 0] * v1[:, 1] - x1[:, 1] * v1[:, 0]).sum() + p.J_body * abs(b1[5])
    assert np.abs(v1).max() > 0.05          # the fluid really moved
    assert np.abs(p1 - p0).max() < 1e-12 * pscale
    assert abs(L1 - L0) < 1e-12 * Lscale
    # mass: the particle set and the particle mass are unchanged by the step
    assert x1.shape == x.shape and np.all(np.isfinite(x1))


def test_interior_density_near_rest_and_partition_of_unity(orc):
    # With the normalised constant, the lattice Riemann sum of Eq. 7 gives the
    # rest density in the interior, and the Shepard sum (A = 1) is 1 there.
    p = orc.params(**W.SMALL)
    x, gB = orc.tank(p)
    out = orc.evaluate(p, x, np.zeros_like(x), gB, np.zeros(6))
    h = orc.h_of(p)
    c = orc.fill_chord(p.R, p.fill)
    interior = (np.hypot(x[:, 0], x[:, 1]) < p.R - 4 * h) & (x[:, 1] < c - 4 * h)
    assert interior.sum() > 300
    np.testing.assert_allclose(out["rho"][interior], p.rho0, rtol=2e-3)
    S = orc.shepard(p, x, out["rho"])
    np.testing.assert_allclose(S[interior], 1.0, atol=1e-12)
    # the printed constant would triple the interior density
    p3 = orc.params(**dict(W.SMALL, sigma_cubic=15.0 / (14.0 * math.pi)))
    out3 = orc.evaluate(p3, x, np.zeros_like(x), gB, np.zeros(6))
    np.testing.assert_allclose(out3["rho"][interior], 3 * p.rho0, rtol=2e-3)


def test_eos_unclamped(orc):
    p = orc.params(**W.SMALL)
    x, gB = orc.tank(p)
    out = orc.evaluate(p, x, np.zeros_like(x), gB, np.zeros(6))
    np.testing.assert_allclose(out["P"], p.k * (out["rho"] - p.rho0), rtol=1e-15, atol=1e-12)
    assert out["P"].min() < 0  # the free surface is under tension


def test_continuity_sum_is_time_derivative_of_density(orc):
    # The continuity sum is read as d rho_i / dt of Eq. 14 along the kinematic
    # motion of fluid (x + t v) and body (pose + t velocity).
    p = orc.params(**W.TINY)
    x, gB = orc.tank(p)
    x = x + W.perturbation(x.shape, 0.2 * p.dx, seed=5)
    v = W.perturbation(x.shape, 0.4, seed=6)
    body = np.array([0.0, 0.0, 0.2, 0.3, -0.2, 1.5])
    out = orc.evaluate(p, x, v, gB, body)
    d = 1e-7
    bp = body.copy(); bp[:3] += d * body[3:]
    bm = body.copy(); bm[:3] -= d * body[3:]
    rp = orc.evaluate(p, x + d * v, v, gB, bp)["rho"]
    rm = orc.evaluate(p, x - d * v, v, gB, bm)["rho"]
    fd = (rp - rm) / (2 * d)
    np.testing.assert_allclose(out["drho"], fd, rtol=0, atol=1e-5 * np.abs(fd).max())


def test_relaxed_fluid_stays_at_rest(orc):
    # Section 5.1: a spawned fluid relaxed to zero velocity without actuation
    # is a steady state; from it, no input keeps fluid and body at rest.
    p = orc.params(**dict(W.TINY, dt=1e-4))
    x, gB = orc.tank(p)
    v = np.zeros_like(x)
    body = np.zeros(6)
    for _ in range(200):
        x, v, body, _, _ = orc.run(p, x, v, gB, body, 1000, damping=5e-3, record=False)
        body[:] = 0.0
        if np.abs(v).max() < 1e-9:
            break
    assert np.abs(v).max() < 1e-8
    p2 = orc.params(**dict(W.TINY, dt=5e-5))
    x2, v2, b2, _, _ = orc.run(p2, x, np.zeros_like(v), gB, np.zeros(6), 2000, record=False)
    assert np.abs(v2).max() < 1e-5
    assert np.abs(b2[3:]).max() < 1e-5
    assert np.abs(b2[:3]).max() < 1e-9


# --------------------------------------------------------------------------
# rigid body and controller (no fluid)
# --------------------------------------------------------------------------
def test_body_under_constant_force_discrete_closed_form(orc):
    # Eq. 20 with no fluid and kick-then-drift: v_n = n dt a, r_n = dt^2 a n(n+1)/2.
    p = orc.params(**dict(W.SMALL, dt=1e-3))
    n = 137
    u = np.tile([2.0, -3.0, 0.5], (n, 1))
    _, _, b, _, _ = orc.run(p, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(6), n, u=u,
                            record=False)
    a = np.array([2.0 / p.m_body, -3.0 / p.m_body, 0.5 / p.J_body])
    np.testing.assert_allclose(b[3:], n * p.dt * a, rtol=1e-13)
    np.testing.assert_allclose(b[:3], p.dt**2 * a * n * (n + 1) / 2, rtol=1e-13)


def test_pd_attitude_controller_matches_second_order_response(orc):
    # Eq. 28 with K = [J w^2, 2 xi J w] on a rigid body closes a loop with
    # natural frequency w and damping xi; a fine ZOH tracks the continuous
    # unit-step response.
    p = orc.params(**dict(W.SMALL, dt=1e-3, outer_every=5))
    n = 20000
    ref = np.ones(n // 5)
    _, _, _, y, _ = orc.run(p, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(6), n,
                            theta_ref=ref, use_ctrl=True)
    t = np.arange(y.shape[0]) * 5 * p.dt
    w, xi = p.ctrl_omega, p.ctrl_xi
    wd = w * math.sqrt(1 - xi * xi)
    theta = 1 - np.exp(-xi * w * t) * (np.cos(wd * t) + xi / math.sqrt(1 - xi * xi) * np.sin(wd * t))
    np.testing.assert_allclose(y[:, 2], theta, atol=5e-3)

"""Plain FP64 NumPy oracle of the self-scheduled LPV surrogate of Section 4
as identified in Section 5.3.2, with its integrator augmentation and its use
in closed loop (Sections 5.1.1 and 5.4).

TEST INFRASTRUCTURE ONLY: used by tests/, never by the product path; it
shares no code with the CUDA library.

Model (Eqs. 24, 25 with the scheduling map of Section 4; n_p = 1, D = 0):
    z_k = [x_k; u_k],  p_k = eta(z_k),
    eta(z) = w3 . tanh(W2 tanh(W1 z + b1) + b2) + b3     (two hidden tanh layers)
    M(p) = M_0 + p M_1 = [[A(p), B(p)], [C(p), 0]],
    x_{k+1} = A(p_k) x_k + B(p_k) u_k,   y_k = C(p_k) x_k.
The parameters are held as a dict of arrays (see `unpack`) and as one flat
vector theta in the order M_0, M_1 (row-major, shape (nx+ny, nx+nu), the D
blocks included but held at zero), W1, b1, W2, b2, w3, b3.

Loss (Eqs. 4, 26, 27): the mean over all samples of ||y_k - y_hat_k||^2
plus sigma2/2 ||theta||^2.  x_0 = 0: every trajectory starts at rest, so the
sigma_x term of Eq. 27 vanishes.
"""
from __future__ import annotations

import numpy as np


def sizes(nx, nu, ny, nh=4):
    """Block sizes of theta in order (M0, M1, W1, b1, W2, b2, w3, b3)."""
    nm = (nx + ny) * (nx + nu)
    nz = nx + nu
    return [nm, nm, nh * nz, nh, nh * nh, nh, nh, 1]


def unpack(theta, nx, nu, ny, nh=4):
    s = np.cumsum([0] + sizes(nx, nu, ny, nh))
    nz = nx + nu
    P = {}
    P["M0"] = theta[s[0]:s[1]].reshape(nx + ny, nz)
    P["M1"] = theta[s[1]:s[2]].reshape(nx + ny, nz)
    P["W1"] = theta[s[2]:s[3]].reshape(nh, nz)
    P["b1"] = theta[s[3]:s[4]]
    P["W2"] = theta[s[4]:s[5]].reshape(nh, nh)
    P["b2"] = theta[s[5]:s[6]]
    P["w3"] = theta[s[6]:s[7]]
    P["b3"] = theta[s[7]:s[8]]
    return P


def pack(P):
    return np.concatenate([P[k].ravel() for k in ("M0", "M1", "W1", "b1", "W2", "b2", "w3", "b3")])


def d_mask(nx, nu, ny, nh=4):
    """1 for every trainable entry, 0 on the feedthrough blocks D of M_0, M_1."""
    m = np.ones(sum(sizes(nx, nu, ny, nh)))
    nz = nx + nu
    for blk in range(2):
        M = np.ones((nx + ny, nz))
        M[nx:, nx:] = 0.0
        m[blk * (nx + ny) * nz:(blk + 1) * (nx + ny) * nz] = M.ravel()
    return m


def eta(P, z):
    """Scheduling map (two tanh layers of nh neurons, linear output)."""
    h1 = np.tanh(P["W1"] @ z + P["b1"])
    h2 = np.tanh(P["W2"] @ h1 + P["b2"])
    return float(P["w3"] @ h2 + P["b3"][0]), h1, h2


def simulate(theta, u, nx, ny, x0=None):
    """Free run over u [T, nu]: returns (y_hat [T, ny], x [T+1, nx], p [T])."""
    T, nu = u.shape
    P = unpack(theta, nx, nu, ny)
    x = np.zeros(nx) if x0 is None else np.array(x0, dtype=np.float64)
    xs = np.zeros((T + 1, nx))
    ys = np.zeros((T, ny))
    ps = np.zeros(T)
    xs[0] = x
    for k in range(T):
        z = np.concatenate([x, u[k]])
        p, _, _ = eta(P, z)
        M = P["M0"] + p * P["M1"]
        o = M @ z
        ys[k] = o[nx:]
        x = o[:nx]
        xs[k + 1] = x
        ps[k] = p
    return ys, xs, ps


def loss(theta, U, Y, nx, sigma2):
    ny = Y[0].shape[1]
    tot, n = 0.0, 0
    for u, y in zip(U, Y):
        yh, _, _ = simulate(theta, u, nx, ny)
        tot += np.sum((y - yh) ** 2)
        n += y.shape[0]
    return tot / n + 0.5 * sigma2 * np.sum(theta * theta)


def loss_grad(theta, U, Y, nx, sigma2, mask=None):
    """Gradient of `loss` by backpropagation through time, through the state
    recursion and through the scheduling map (which depends on the state)."""
    nu, ny = U[0].shape[1], Y[0].shape[1]
    P = unpack(theta, nx, nu, ny)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    n = sum(y.shape[0] for y in Y)
    for u, y in zip(U, Y):
        T = u.shape[0]
        yh, xs, ps = simulate(theta, u, nx, ny)
        lam = np.zeros(nx)                                   # dJ/dx_{k+1}
        for k in range(T - 1, -1, -1):
            z = np.concatenate([xs[k], u[k]])
            p, h1, h2 = eta(P, z)
            a = np.concatenate([lam, 2.0 * (yh[k] - y[k]) / n])  # dJ/d[x_{k+1}; y_k]
            M = P["M0"] + p * P["M1"]
            G["M0"] += np.outer(a, z)
            G["M1"] += p * np.outer(a, z)
            s = float(a @ (P["M1"] @ z))                     # dJ/dp_k
            # back through eta
            G["w3"] += s * h2
            G["b3"] += s
            d2 = s * P["w3"] * (1.0 - h2 * h2)
            G["W2"] += np.outer(d2, h1)
            G["b2"] += d2
            d1 = (P["W2"].T @ d2) * (1.0 - h1 * h1)
            G["W1"] += np.outer(d1, z)
            G["b1"] += d1
            dz = M.T @ a + P["W1"].T @ d1                     # dJ/dz_k
            lam = dz[:nx]
    g = pack(G) + sigma2 * theta
    if mask is not None:
        g = g * mask
    return g


def augment(theta, u, nx, ny, Ts):
    """Integrator augmentation (the full surrogate after Section 5.3.2):
    e_{k+1} = e_k + Ts (C(p_k) x_k + D(p_k) u_k) with D = 0, e_0 = 0; returns
    the positions e [T, ny] (before each step) and velocities y_hat [T, ny]."""
    yh, _, _ = simulate(theta, u, nx, ny)
    e = np.zeros_like(yh)
    e[1:] = Ts * np.cumsum(yh[:-1], axis=0)
    return e, yh


def closed_loop(theta, nx, scales, F, tau, theta_ref, Ts, pd):
    """Closed loop of the augmented surrogate with the PD law of Eq. 28.

    The model maps u = [F_x, F_y, tau] to the velocities [rdot_x, rdot_y,
    thetadot] in normalised units (u / s_u, y * s_y).  At sample k the
    controller reads theta_k (augmented state) and thetadot_k = C(p) x_k with
    p = eta(x_k, u_{k-1}), the input held when the sample is taken (u_{-1} = 0);
    then u_k = [F_k, tau_k + tau_c,k] is applied, p_k = eta(x_k, u_k) and
    x_{k+1} = A(p_k) x_k + B(p_k) u_k, e_{k+1} = e_k + Ts C(p_k) x_k.
    Returns [T, 6] samples (r_x, r_y, theta, rdot_x, rdot_y, thetadot), where
    the velocities are C(p_k) x_k of the step."""
    nu, ny = 3, 3
    P = unpack(theta, nx, nu, ny)
    su, sy = np.asarray(scales["u"], float), np.asarray(scales["y"], float)
    J, w, xi = pd["J"], pd["omega"], pd["xi"]
    T = F.shape[0]
    x = np.zeros(nx)
    e = np.zeros(3)
    un_prev = np.zeros(nu)
    out = np.zeros((T, 6))
    for k in range(T):
        zm = np.concatenate([x, un_prev])
        pm, _, _ = eta(P, zm)
        ym = ((P["M0"] + pm * P["M1"]) @ zm)[nx:] * sy
        tc = J * w * w * (theta_ref[k] - e[2]) - 2.0 * xi * J * w * ym[2]
        un = np.array([F[k, 0], F[k, 1], tau[k] + tc]) / su
        z = np.concatenate([x, un])
        p, _, _ = eta(P, z)
        o = (P["M0"] + p * P["M1"]) @ z
        yv = o[nx:] * sy
        out[k, :3] = e
        out[k, 3:] = yv
        e = e + Ts * yv
        x = o[:nx]
        un_prev = un
    return out


def ls_start(U, Y, nx):
    """Least-squares LTI start of M_0 (stands in for the ssest fit of Section
    5.3.2): the first-order ARX model y_{k+1} = A1 y_k + B1 u_k fitted by the
    normal equations over all samples of all trajectories (normalised data),
    realised with the velocities as the first three states: A_0 = [[A1, 0],
    [0, 0]], B_0 = [[B1], [0]], C_0 = [I, 0]; M_1 and the network zero."""
    ny, nu = Y[0].shape[1], U[0].shape[1]
    Phi = np.concatenate([np.concatenate([y[:-1], u[:-1]], axis=1) for u, y in zip(U, Y)])
    Tgt = np.concatenate([y[1:] for y in Y])
    G = Phi.T @ Phi
    R = Phi.T @ Tgt
    Th = np.linalg.solve(G + 1e-12 * np.trace(G) / G.shape[0] * np.eye(G.shape[0]), R)   # [ny+nu, ny]
    A1, B1 = Th[:ny].T, Th[ny:].T
    P = unpack(np.zeros(sum(sizes(nx, nu, ny))), nx, nu, ny)
    P["M0"][:ny, :ny] = A1
    P["M0"][:ny, nx:] = B1
    P["M0"][nx:, :ny] = np.eye(ny)
    return pack(P)

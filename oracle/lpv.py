"""Plain FP64 NumPy oracle of the LPV surrogate (Section 4) and of its use in
closed loop (Sections 5.1.1 and 5.4).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU baseline, never
by the product path; it shares no code with the CUDA library.

Model (Eqs. 24, 25; feedthrough D fixed to zero as in Section 5.3.2):
    x_{k+1} = A(p_k) x_k + B(p_k) u_k,   y_k = C(p_k) x_k,
    M(p) = [[A, B], [C, D]] = M_0 + sum_i p_i M_i.
Parameters are stored as W = [M_0, M_1, ..., M_np], shape (nx+ny, (1+np)(nx+nu)),
so that [x_{k+1}; y_k] = W @ w_k with w_k = [z_k; p_1 z_k; ...], z_k = [x_k; u_k].
The scheduling p is an input of the model here (fill fraction and body
angular rate), so no network eta is learned.

Loss (Eqs. 4, 26, 27): the mean squared free-run simulation error over all
trajectories and samples plus sigma2/2 ||theta||^2, with x_0 = 0 (the fluid
starts at rest, Section 2.2), so the sigma_x term vanishes.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# model
# --------------------------------------------------------------------------
def features(x, u, p):
    """w = [z, p_1 z, ..., p_np z] with z = [x, u] (Eq. 25)."""
    z = np.concatenate([x, u])
    return np.concatenate([z] + [pi * z for pi in p])


def simulate(W, u, p, nx, x0=None):
    """Free-run simulation of Eq. 24: returns y_hat [T, ny] and x [T+1, nx]."""
    T = u.shape[0]
    ny = W.shape[0] - nx
    x = np.zeros(nx) if x0 is None else np.array(x0, dtype=np.float64)
    xs = np.zeros((T + 1, nx))
    ys = np.zeros((T, ny))
    xs[0] = x
    for k in range(T):
        out = W @ features(x, u[k], p[k])
        ys[k] = out[nx:]
        x = out[:nx]
        xs[k + 1] = x
    return ys, xs


def loss(W, U, Y, P, nx, sigma2):
    """J = mean over trajectories and samples of ||y - y_hat||^2 + sigma2/2 ||W||^2."""
    tot = 0.0
    n = 0
    for u, y, p in zip(U, Y, P):
        yh, _ = simulate(W, u, p, nx)
        tot += np.sum((y - yh) ** 2)
        n += y.shape[0]
    return tot / n + 0.5 * sigma2 * np.sum(W * W)


def loss_grad(W, U, Y, P, nx, sigma2, mask=None):
    """Gradient of `loss` by backpropagation through time (FP64).
    mask (same shape as W, 0/1) zeroes fixed entries (the D block)."""
    G = np.zeros_like(W)
    n = sum(y.shape[0] for y in Y)
    for u, y, p in zip(U, Y, P):
        T = u.shape[0]
        yh, xs = simulate(W, u, p, nx)
        lam = np.zeros(nx)                         # dJ/dx_{k+1}
        for k in range(T - 1, -1, -1):
            g = np.concatenate([lam, 2.0 * (yh[k] - y[k]) / n])   # dJ/d[x_{k+1}; y_k]
            w = features(xs[k], u[k], p[k])
            G += np.outer(g, w)
            gw = W.T @ g                           # dJ/dw_k
            nz = nx + u.shape[1]
            lam = gw[:nx].copy()
            for i, pi in enumerate(p[k]):
                lam += pi * gw[(i + 1) * nz:(i + 1) * nz + nx]
    G += sigma2 * W
    if mask is not None:
        G = G * mask
    return G


def d_mask(nx, nu, ny, n_p):
    """1 everywhere except the feedthrough blocks D of every M_i."""
    m = np.ones((nx + ny, (1 + n_p) * (nx + nu)))
    for i in range(1 + n_p):
        m[nx:, i * (nx + nu) + nx:(i + 1) * (nx + nu)] = 0.0
    return m


# --------------------------------------------------------------------------
# FP64 least-squares initialisation of M_0 (replaces the LTI ssest fit)
# --------------------------------------------------------------------------
def arx_ls(U, Y, na, nb):
    """MIMO ARX y_k = sum_{i=1..na} A_i y_{k-i} + sum_{i=1..nb} B_i u_{k-i}
    fitted by the normal equations over all trajectories; returns (A_i), (B_i)."""
    ny, nu = Y[0].shape[1], U[0].shape[1]
    rows, targ = [], []
    m = max(na, nb)
    for u, y in zip(U, Y):
        for k in range(m, y.shape[0]):
            rows.append(np.concatenate([y[k - i] for i in range(1, na + 1)] + [u[k - i] for i in range(1, nb + 1)]))
            targ.append(y[k])
    Phi = np.array(rows)
    Yt = np.array(targ)
    theta = np.linalg.solve(Phi.T @ Phi, Phi.T @ Yt)        # [na*ny + nb*nu, ny]
    A = [theta[(i - 1) * ny:i * ny].T for i in range(1, na + 1)]
    B = [theta[na * ny + (i - 1) * nu:na * ny + i * nu].T for i in range(1, nb + 1)]
    return A, B


def arx_to_ss(A, B):
    """Observer-canonical state space of the ARX model (na = nb = n):
    x^j_{k+1} = A_j y_k + x^{j+1}_k + B_j u_k,  y_k = x^1_k."""
    n = len(A)
    ny, nu = B[0].shape
    nx = n * ny
    As = np.zeros((nx, nx))
    Bs = np.zeros((nx, nu))
    for j in range(n):
        As[j * ny:(j + 1) * ny, 0:ny] = A[j]
        if j + 1 < n:
            As[j * ny:(j + 1) * ny, (j + 1) * ny:(j + 2) * ny] = np.eye(ny)
        Bs[j * ny:(j + 1) * ny] = B[j]
    Cs = np.zeros((ny, nx))
    Cs[:, :ny] = np.eye(ny)
    return As, Bs, Cs


def stabilize(A, B, rho_max):
    """Stable LTI start (the paper starts from a stable identified model): if
    the spectral radius rho of the observer-canonical state matrix exceeds
    rho_max, every characteristic root is scaled by lam = rho_max / rho via
    A_i <- lam^i A_i, B_i <- lam^i B_i (impulse response h_k -> lam^k h_k).
    Returns (A, B, rho)."""
    As, _, _ = arx_to_ss(A, B)
    rho = float(np.max(np.abs(np.linalg.eigvals(As)))) if As.size else 0.0
    if rho_max <= 0 or rho <= rho_max:
        return [a.copy() for a in A], [b.copy() for b in B], rho
    lam = rho_max / rho
    return ([lam ** (i + 1) * a for i, a in enumerate(A)], [lam ** (i + 1) * b for i, b in enumerate(B)], rho)


def balance(As, Bs, Cs, reg=1e-12):
    """Balanced realisation (Moore 1981) of a stable (A, B, C), the form in
    which the least-squares start is handed to training: with the Gramians
    P = A P A^T + B B^T and Q = A^T Q A + C^T C (each regularised by
    reg * trace * I), P = Lp Lp^T, Q = Lq Lq^T and Lq^T Lp = U S V^T,
    T = Lp V S^(-1/2) and T^-1 = S^(-1/2) U^T Lq^T give (T^-1 A T, T^-1 B, C T),
    whose Gramians both equal diag(S).  States are ordered by decreasing S and
    signed so that the largest-magnitude entry of each column of C T is
    positive.  Returns (A, B, C, S)."""
    import scipy.linalg as sl

    n = As.shape[0]
    P = sl.solve_discrete_lyapunov(As, Bs @ Bs.T)
    Q = sl.solve_discrete_lyapunov(As.T, Cs.T @ Cs)
    P = P + reg * np.trace(P) * np.eye(n)
    Q = Q + reg * np.trace(Q) * np.eye(n)
    Lp = np.linalg.cholesky(P)
    Lq = np.linalg.cholesky(Q)
    U, S, Vt = np.linalg.svd(Lq.T @ Lp)
    T = Lp @ Vt.T / np.sqrt(S)
    Ti = (U / np.sqrt(S)).T @ Lq.T
    Ab, Bb, Cb = Ti @ As @ T, Ti @ Bs, Cs @ T
    sign = np.sign(Cb[np.argmax(np.abs(Cb), axis=0), np.arange(n)])
    sign[sign == 0] = 1.0
    return sign[:, None] * Ab * sign[None, :], sign[:, None] * Bb, Cb * sign[None, :], S


def ss_to_W(As, Bs, Cs, n_p):
    """W = [M_0, 0, ..., 0] with M_0 = [[A, B], [C, 0]]."""
    nx, nu = Bs.shape
    ny = Cs.shape[0]
    M0 = np.zeros((nx + ny, nx + nu))
    M0[:nx, :nx] = As
    M0[:nx, nx:] = Bs
    M0[nx:, :nx] = Cs
    return np.concatenate([M0] + [np.zeros_like(M0)] * n_p, axis=1)


def ls_start(U, Y, na, rho_max, n_p):
    """The least-squares start W = [M_0, 0, ..]: ARX fit, roots scaled into
    |z| <= rho_max, observer-canonical form, balanced when 0 < rho_max < 1."""
    A, B = arx_ls(U, Y, na, na)
    A, B, _ = stabilize(A, B, rho_max)
    As, Bs, Cs = arx_to_ss(A, B)
    if 0.0 < rho_max < 1.0:
        As, Bs, Cs, _ = balance(As, Bs, Cs)
    return ss_to_W(As, Bs, Cs, n_p)


# --------------------------------------------------------------------------
# Adam (Kingma and Ba), used by the paper before L-BFGS (Section 4)
# --------------------------------------------------------------------------
def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at iteration t >= 1; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# closed loop: rigid body + surrogate sloshing loads + PD attitude control
# --------------------------------------------------------------------------
def closed_loop(W, nx, scales, body, fill, F, tau, theta_ref, Ts, n_sub, pd, p_range=None):
    """One closed-loop run at the sampling period Ts (Section 5.1.1):
      tau_c,k = J w^2 (theta_ref_k - theta_k) - 2 xi J w thetadot_k   (Eq. 28, ZOH)
      u_k = [F_x, F_y, tau + tau_c],  p_k = [fill, thetadot_k][:n_p]
      surrogate (normalised units): y_k = C(p) x_k, x_{k+1} = A(p) x_k + B(p) u_k
      sloshing loads [F_bx, F_by, T_b] = y_k[:3] * y_scale[:3]
      body (Eq. 20 with the loads held over the period): n_sub kick-then-drift
      substeps of Ts / n_sub.
    scales: dict(u, y, p_mean, p_scale).  p_range (lo, hi), if given: p is
    clamped to it (the range the model was identified on) before scaling.
    Returns [T, 6] samples (before each period) of r_x, r_y, theta, rdot_x,
    rdot_y, thetadot."""
    m, J = body["m"], body["J"]
    Jc = pd.get("J", J) if pd.get("J", 0) > 0 else J
    w, xi = pd["omega"], pd["xi"]
    T = F.shape[0]
    x = np.zeros(nx)
    s = np.zeros(6)   # r_x r_y theta v_x v_y omega
    out = np.zeros((T, 6))
    dt = Ts / n_sub
    n_p = W.shape[1] // (nx + 3) - 1
    for k in range(T):
        out[k] = s
        tc = Jc * w * w * (theta_ref[k] - s[2]) - 2.0 * xi * Jc * w * s[5]
        u = np.array([F[k, 0], F[k, 1], tau[k] + tc])
        p = np.array([fill, s[5]])[:n_p]
        if p_range is not None:
            p = np.minimum(np.maximum(p, p_range[0]), p_range[1])
        p = (p - scales["p_mean"]) / scales["p_scale"]
        o = W @ features(x, u / scales["u"], p)
        x = o[:nx]
        yl = o[nx:] * scales["y"]
        ax, ay, aw = (u[0] + yl[0]) / m, (u[1] + yl[1]) / m, (u[2] + yl[2]) / J
        for _ in range(n_sub):
            s[3] += dt * ax
            s[4] += dt * ay
            s[5] += dt * aw
            s[0] += dt * s[3]
            s[1] += dt * s[4]
            s[2] += dt * s[5]
    return out


def bfr(y, yh):
    """Best fit rate per channel (footnote in Section 5.3.2), in percent."""
    num = np.sqrt(np.sum((y - yh) ** 2, axis=0))
    den = np.sqrt(np.sum((y - y.mean(axis=0)) ** 2, axis=0))
    return 100.0 * (1.0 - num / den)

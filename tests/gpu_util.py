"""Helpers shared by the GPU tests (no arithmetic of the method)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12505_gb300 import build
    build.build()
    return torch


def oracle_state(orc, cfg, pos_sigma=0.0, vel_sigma=0.0, seed=0):
    """Oracle tank + seeded perturbation, rounded to the FP32 state the GPU
    holds; returns (xv float32 [N, 4], x64, v64) with x64/v64 the exact FP64
    values of the FP32 numbers."""
    from paper_2604_12505_gb300 import workloads as W
    p = orc.params(**cfg)
    x, gB = orc.tank(p)
    if pos_sigma:
        x = x + W.perturbation(x.shape, pos_sigma * cfg["dx"], seed=seed)
    v = W.perturbation(x.shape, vel_sigma, seed=seed + 1) if vel_sigma else np.zeros_like(x)
    xv = np.concatenate([x, v], axis=1).astype(np.float32)
    return xv, xv[:, :2].astype(np.float64), xv[:, 2:].astype(np.float64), gB, p


def normwise(a, b):
    """max |a - b| / max |b| (row-wise norms for 2-D arrays)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 2:
        num, den = np.linalg.norm(a - b, axis=1).max(), np.linalg.norm(b, axis=1).max()
    else:
        num, den = np.abs(a - b).max(), np.abs(b).max()
    if den == 0.0:  # an all-zero reference must be matched exactly
        return 0.0 if num == 0.0 else np.inf
    return num / den


# Groups of the output record compared as vectors: body position, angle,
# body velocity, angular rate, fluid centre of mass.
TRAJ_GROUPS = {"r": [0, 1], "theta": [2], "rdot": [3, 4], "thetadot": [5], "com": [9, 10]}


def traj_err(yg, yr):
    """Per group: max_t ||q_gpu(t) - q_ref(t)|| / max_t ||q_ref(t)||."""
    out = {}
    for name, cols in TRAJ_GROUPS.items():
        d = np.linalg.norm(yg[:, cols] - yr[:, cols], axis=1).max()
        out[name] = d / np.linalg.norm(yr[:, cols], axis=1).max()
    return out


def body_force_tolerance(ev, e_rho, rel=1e-5):
    """Bound on |F_gpu - F_ref| per component (F_x, F_y, T_b) from the
    arithmetic: the fluid-ghost pair forces that make up the body force carry
    the error of their particle's density (e_rho, the measured maximum
    relative density error) through Eq. 11, which the oracle's fb_drho sums as
    rho df/drho over the pairs, plus FP32 rounding of each pair term, at most
    ``rel`` of its magnitude (fb_abs)."""
    return e_rho * np.asarray(ev["fb_drho"]) + rel * np.asarray(ev["fb_abs"]) + 1e-12

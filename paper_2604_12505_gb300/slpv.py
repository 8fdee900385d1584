"""Python front end of the self-scheduled LPV surrogate of Section 5.3.2
(argument marshalling only; every computation runs in the CUDA library, see
``include/slpv.h``).

The model maps the applied input u = [F_x, F_y, tau] to the body velocities
[rdot_x, rdot_y, thetadot] at the sampling period T_s; its scheduling p is
computed from the state and the input by a small tanh network, and the
positions are recovered by the integrator augmentation.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .sph import _dev, _ptr, _stream


class SlpvConfig(C.Structure):
    _fields_ = [("nx", C.c_int32), ("sigma2", C.c_float)]


def n_params(nx: int) -> int:
    n = C.c_int32()
    check(lib().slpv_n_params(nx, C.byref(n)), "slpv_n_params")
    return n.value


class VelocityModel:
    """A self-scheduled LPV model held by the CUDA library."""

    def __init__(self, nx: int = 4, sigma2: float = 1e-4):
        self.nx = nx
        self.sigma2 = sigma2
        cfg = SlpvConfig(nx, sigma2)
        h = C.c_void_p()
        check(lib().slpv_create(C.byref(cfg), C.byref(h)), "slpv_create")
        self._h = h
        self.n = n_params(nx)

    def close(self):
        if self._h:
            lib().slpv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters ----------------------------------------------------------
    def set_params(self, theta=None, scales=None):
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        if th is not None and th.size != self.n:
            raise ValueError(f"theta needs {self.n} values")
        check(lib().slpv_set_params(self._h, None if th is None else th.ctypes.data,
                                    None if sc is None else sc.ctypes.data), "slpv_set_params")

    def get_params(self):
        th = np.zeros(self.n, dtype=np.float32)
        sc = np.zeros(6, dtype=np.float32)
        check(lib().slpv_get_params(self._h, th.ctypes.data, sc.ctypes.data), "slpv_get_params")
        return th, sc

    # -- data ------------------------------------------------------------------
    @staticmethod
    def _data(t):
        t = _dev(t, torch.float32)
        if t.dim() != 3 or t.shape[2] != 3:
            raise ValueError("expected [n_traj, T, 3]")
        return t

    def normalize(self, u, y, stream=None):
        u, y = self._data(u), self._data(y)
        check(lib().slpv_normalize(self._h, _ptr(u), _ptr(y), u.shape[0], u.shape[1], _stream(stream)),
              "slpv_normalize")

    def init_ls(self, u, y, stream=None):
        """Least-squares LTI start of M_0 (first-order ARX on the scaled data)."""
        u, y = self._data(u), self._data(y)
        check(lib().slpv_init_ls(self._h, _ptr(u), _ptr(y), u.shape[0], u.shape[1], _stream(stream)),
              "slpv_init_ls")

    # training stages: which entries of theta move
    ALL, LTI, SCHEDULING = 0, 1, 2

    def loss_grad(self, u, y, stage: int = 0, grad: bool = True, stream=None):
        u, y = self._data(u), self._data(y)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.zeros(self.n, dtype=torch.float32, device="cuda") if grad else None
        check(lib().slpv_loss_grad(self._h, _ptr(u), _ptr(y), u.shape[0], u.shape[1], stage, _ptr(loss),
                                   _ptr(g), _stream(stream)), "slpv_loss_grad")
        return loss, g

    def train(self, u, y, iters: int, lr: float, stage: int = 0, stream=None):
        """Adam steps on the entries of `stage`; returns the loss at every
        iterate (device float64 [iters])."""
        u, y = self._data(u), self._data(y)
        hist = torch.zeros(max(iters, 1), dtype=torch.float64, device="cuda")
        check(lib().slpv_train(self._h, _ptr(u), _ptr(y), u.shape[0], u.shape[1], iters, lr, stage,
                               _ptr(hist), _stream(stream)), "slpv_train")
        return hist[:iters]

    def lbfgs(self, u, y, iters: int, stage: int = 0, stream=None):
        """L-BFGS iterations; returns the accepted loss per iteration (host)."""
        u, y = self._data(u), self._data(y)
        hist = np.zeros(max(iters, 1), dtype=np.float64)
        check(lib().slpv_lbfgs(self._h, _ptr(u), _ptr(y), u.shape[0], u.shape[1], iters, stage,
                               hist.ctypes.data, _stream(stream)), "slpv_lbfgs")
        return hist[:iters]

    # -- use ---------------------------------------------------------------------
    def predict(self, u, Ts: float, stream=None):
        """Free run from rest: (velocities, positions), each [n_traj, T, 3]."""
        u = self._data(u)
        vel = torch.empty_like(u)
        pos = torch.empty_like(u)
        check(lib().slpv_predict(self._h, _ptr(u), u.shape[0], u.shape[1], Ts, _ptr(vel), _ptr(pos),
                                 _stream(stream)), "slpv_predict")
        return vel, pos

    def simulate(self, F, tau, theta_ref, Ts: float, J: float, omega: float, xi: float, stream=None):
        """Closed loop under the PD law of Eq. 28: [B, T, 6] rows (r_x, r_y,
        theta, rdot_x, rdot_y, thetadot)."""
        F = _dev(F, torch.float64)
        tau = _dev(tau, torch.float64)
        ref = _dev(theta_ref, torch.float64)
        B, T = tau.shape
        if F.shape != (B, T, 2) or ref.shape != (B, T):
            raise ValueError("F [B, T, 2], tau and theta_ref [B, T]")
        out = torch.empty((B, T, 6), dtype=torch.float32, device="cuda")
        check(lib().slpv_simulate(self._h, B, T, _ptr(F), _ptr(tau), _ptr(ref), Ts, J, omega, xi, _ptr(out),
                                  _stream(stream)), "slpv_simulate")
        return out


def layout(nx: int) -> dict:
    """Slices of theta: M0, M1 ((nx+3) x (nx+3) each), W1, b1, W2, b2, w3, b3."""
    nz = no = nx + 3
    sizes = [("M0", no * nz), ("M1", no * nz), ("W1", 4 * nz), ("b1", 4), ("W2", 16), ("b2", 4), ("w3", 4), ("b3", 1)]
    out, o = {}, 0
    for k, n in sizes:
        out[k] = slice(o, o + n)
        o += n
    return out


def initial_theta(nx: int, seed: int, base=None, m1_std: float = 1e-2, a0: float = 0.9,
                  bc_std: float = 0.1, net_scale: float = 1.0) -> np.ndarray:
    """Starting point of a fit (Section 5.3.2).  Without `base` (an LTI
    start drawn at random; the least-squares start is ``init_ls``): A_0 =
    a0 I, B_0 and C_0 ~ N(0, bc_std^2), everything else zero.
    With `base` (an LPV restart): M_0 from base; the B and C blocks of M_1
    ~ N(0, m1_std^2) and its A block zero, so that A(p) = A_0 keeps the start's
    spectrum; network weights by Xavier's uniform rule (scaled by net_scale),
    biases zero."""
    rng = np.random.default_rng(seed)
    L = layout(nx)
    nz = nx + 3
    th = np.zeros(L["b3"].stop, dtype=np.float64)
    if base is None:
        M0 = np.zeros((nz, nz))
        M0[:nx, :nx] = a0 * np.eye(nx)
        M0[:nx, nx:] = rng.normal(0.0, bc_std, (nx, 3))
        M0[nx:, :nx] = rng.normal(0.0, bc_std, (3, nx))
        th[L["M0"]] = M0.ravel()
        return th.astype(np.float32)
    th[:] = np.asarray(base, dtype=np.float64)
    M1 = np.zeros((nz, nz))
    M1[:nx, nx:] = rng.normal(0.0, m1_std, (nx, 3))
    M1[nx:, :nx] = rng.normal(0.0, m1_std, (3, nx))
    th[L["M1"]] = M1.ravel()
    for name, fan_in, fan_out in (("W1", nz, 4), ("W2", 4, 4), ("w3", 4, 1)):
        lim = net_scale * np.sqrt(6.0 / (fan_in + fan_out))
        th[L[name]] = rng.uniform(-lim, lim, L[name].stop - L[name].start)
    th[L["b1"]] = th[L["b2"]] = th[L["b3"]] = 0.0
    return th.astype(np.float32)

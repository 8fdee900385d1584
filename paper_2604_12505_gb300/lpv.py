"""Python front end of the LPV surrogate (argument marshalling only; every
computation runs in the CUDA library, see ``include/lpv.h``)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .sph import _dev, _ptr, _stream


class LpvConfig(C.Structure):
    """Mirror of ``lpv_config`` (96 bytes, field order matters)."""

    _fields_ = [
        ("n_x", C.c_int32), ("n_u", C.c_int32), ("n_y", C.c_int32), ("n_p", C.c_int32), ("na", C.c_int32),
        ("adam_iters", C.c_int32), ("restarts", C.c_int32), ("lbfgs_iters", C.c_int32),
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("adam_eps", C.c_double),
        ("sigma2", C.c_double), ("init_scale", C.c_double), ("seed", C.c_uint64), ("rho_max", C.c_double),
    ]


class LpvBody(C.Structure):
    _fields_ = [
        ("m", C.c_double), ("J", C.c_double), ("Ts", C.c_double), ("n_sub", C.c_int32), ("reserved", C.c_int32),
        ("ctrl_J", C.c_double), ("ctrl_omega", C.c_double), ("ctrl_xi", C.c_double),
    ]


DEFAULT = dict(n_x=12, n_u=3, n_y=4, n_p=2, na=3, adam_iters=2000, restarts=8, lbfgs_iters=0, lr=1e-3, beta1=0.9, beta2=0.999,
               adam_eps=1e-8, sigma2=1e-4, init_scale=1e-2, seed=7, rho_max=0.999)


def _vp(struct):
    return C.cast(C.pointer(struct), C.c_void_p)


def make_config(d: dict | None = None) -> LpvConfig:
    c = LpvConfig()
    for k, v in dict(DEFAULT, **(d or {})).items():
        setattr(c, k, v)
    return c


class Model:
    """An LPV surrogate held by the CUDA library."""

    def __init__(self, cfg: dict | None = None, _handle=None):
        self.cfg = dict(DEFAULT, **(cfg or {}))
        if _handle is None:
            h = C.c_void_p()
            cfgs = make_config(self.cfg)
            check(lib().lpv_create(_vp(cfgs), C.byref(h)), "lpv_create")
            _handle = h
        self._h = _handle
        c = self.cfg
        self.shape_W = (1 + c["n_p"], c["n_x"] + c["n_y"], c["n_x"] + c["n_u"])
        self.n_scales = c["n_u"] + c["n_y"] + 4 * c["n_p"]

    def close(self):
        if getattr(self, "_h", None):
            lib().lpv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters ----------------------------------------------------------
    def get_params(self):
        W = np.zeros(self.shape_W, dtype=np.float32)
        s = np.zeros(self.n_scales, dtype=np.float32)
        check(lib().lpv_get_params(self._h, W.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p)),
              "lpv_get_params")
        return W, s

    def set_params(self, W=None, scales=None):
        Wc = None if W is None else np.ascontiguousarray(W, dtype=np.float32).reshape(self.shape_W)
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        check(lib().lpv_set_params(self._h, None if Wc is None else Wc.ctypes.data_as(C.c_void_p),
                                   None if sc is None else sc.ctypes.data_as(C.c_void_p)), "lpv_set_params")

    # -- data-driven steps -------------------------------------------------------
    def _data(self, u, y, p):
        u = _dev(u, torch.float32)
        y = None if y is None else _dev(y, torch.float32)
        p = None if p is None else _dev(p, torch.float32)
        return u, y, p, int(u.shape[0]), int(u.shape[1])

    def normalize(self, u, y, p, stream=None):
        u, y, p, n, T = self._data(u, y, p)
        check(lib().lpv_normalize(self._h, _ptr(u), _ptr(y), _ptr(p), n, T, _stream(stream)), "lpv_normalize")

    def init_ls(self, u, y, stream=None):
        u, y, _, n, T = self._data(u, y, None)
        c = self.cfg
        theta = np.zeros((c["na"] * (c["n_y"] + c["n_u"]), c["n_y"]))
        check(lib().lpv_init_ls(self._h, _ptr(u), _ptr(y), n, T, theta.ctypes.data_as(C.c_void_p),
                                _stream(stream)), "lpv_init_ls")
        return theta

    def loss_grad(self, u, y, p, stream=None):
        u, y, p, n, T = self._data(u, y, p)
        loss = C.c_double()
        g = np.zeros(self.shape_W, dtype=np.float32)
        check(lib().lpv_loss_grad(self._h, _ptr(u), _ptr(y), _ptr(p), n, T, C.byref(loss),
                                  g.ctypes.data_as(C.c_void_p), _stream(stream)), "lpv_loss_grad")
        return loss.value, g

    def train(self, u, y, p, iters: int, stream=None):
        u, y, p, n, T = self._data(u, y, p)
        hist = np.zeros(max(iters, 1))
        check(lib().lpv_train(self._h, _ptr(u), _ptr(y), _ptr(p), n, T, iters, hist.ctypes.data_as(C.c_void_p),
                              _stream(stream)), "lpv_train")
        return hist[:iters]

    def lbfgs(self, u, y, p, iters: int, stream=None):
        """L-BFGS iterations from the current weights (lpv_lbfgs); returns the
        accepted loss of each iteration."""
        u, y, p, n, T = self._data(u, y, p)
        hist = np.zeros(max(iters, 1))
        check(lib().lpv_lbfgs(self._h, _ptr(u), _ptr(y), _ptr(p), n, T, iters, hist.ctypes.data_as(C.c_void_p),
                              _stream(stream)), "lpv_lbfgs")
        return hist[:iters]

    def predict(self, u, p, stream=None):
        u, _, p, n, T = self._data(u, None, p)
        y = torch.empty((n, T, self.cfg["n_y"]), dtype=torch.float32, device="cuda")
        check(lib().lpv_predict(self._h, _ptr(u), _ptr(p), n, T, _ptr(y), _stream(stream)), "lpv_predict")
        return y

    def simulate(self, F, tau, theta_ref, fill, body: dict, stream=None):
        """Closed loop of B runs: F [B, T, 2], tau [B, T], theta_ref [B, T],
        fill [B] -> [B, T, 6] body samples (float64, device)."""
        F = _dev(F, torch.float64)
        tau = _dev(tau, torch.float64)
        ref = _dev(theta_ref, torch.float64)
        fill = _dev(fill, torch.float64)
        B, T = int(F.shape[0]), int(F.shape[1])
        b = LpvBody()
        for k in ("m", "J", "Ts", "n_sub", "ctrl_J", "ctrl_omega", "ctrl_xi"):
            setattr(b, k, body.get(k, 0))
        out = torch.empty((B, T, 6), dtype=torch.float64, device="cuda")
        check(lib().lpv_simulate(self._h, B, _ptr(F), _ptr(tau), _ptr(ref), _ptr(fill), T, _vp(b), _ptr(out),
                                 _stream(stream)), "lpv_simulate")
        return out


def fit(u, y, p, cfg: dict | None = None, stream=None):
    """The identification of Section 5.3.2 on device: returns (Model, best loss)."""
    c = dict(DEFAULT, **(cfg or {}))
    u = _dev(u, torch.float32)
    y = _dev(y, torch.float32)
    p = _dev(p, torch.float32)
    h = C.c_void_p()
    best = C.c_double()
    cfgs = make_config(c)
    check(lib().lpv_fit(_ptr(u), _ptr(y), _ptr(p), int(u.shape[0]), int(u.shape[1]), _vp(cfgs),
                        C.byref(h), C.byref(best), _stream(stream)), "lpv_fit")
    return Model(c, _handle=h), best.value

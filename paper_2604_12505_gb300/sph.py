"""Python front end of the SPH sloshing simulator (argument marshalling only).

Every computation runs in the CUDA library through its C ABI; PyTorch only
provides device memory and the current stream.  Parameters are plain dicts
with the fields of ``sph_params`` (see ``include/sph.h``).
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import NY, SphCtrl, SphParams, check, lib

PARAM_FIELDS = [f for f, _ in SphParams._fields_]


def make_params(d: dict) -> SphParams:
    p = SphParams()
    for f in PARAM_FIELDS:
        if f in d:
            setattr(p, f, d[f])
    return p


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype):
    if t is None:
        return None
    t = torch.as_tensor(t, dtype=dtype)
    if t.device.type != "cuda":
        t = t.to("cuda", non_blocking=False)
    return t.contiguous()


def make_ctrl(ctrl: dict | None, theta_ref=None, ref_stride: int = 0) -> SphCtrl | None:
    if not ctrl:
        return None
    c = SphCtrl()
    c.J = ctrl.get("J", 0.0)
    c.omega = ctrl.get("omega", 0.2 * np.pi)
    c.xi = ctrl.get("xi", 0.7)
    c.theta_ref = None if theta_ref is None else theta_ref.data_ptr()
    c.ref_stride = ref_stride
    c.enabled = 1
    return c


class Sim:
    """One tank (dict) or a batch of independent tanks (list of dicts)."""

    def __init__(self, params: dict | Sequence[dict], stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the SPH simulator needs a CUDA device")
        torch.cuda.init()
        plist = [params] if isinstance(params, dict) else list(params)
        arr = (SphParams * len(plist))(*[make_params(d) for d in plist])
        h = C.c_void_p()
        check(lib().sph_create_batch(arr, len(plist), _stream(stream), C.byref(h)), "sph_create")
        self._h = h
        self.params = [dict(d) for d in plist]
        self.B = len(plist)
        nf = (C.c_int32 * self.B)()
        ng = (C.c_int32 * self.B)()
        check(lib().sph_counts(h, None, nf, ng), "sph_counts")
        self.n_fluid = list(nf)
        self.n_ghost = list(ng)
        self.n_total = sum(self.n_fluid)
        self.offsets = np.concatenate([[0], np.cumsum(self.n_fluid)]).astype(int)
        self.steps_done = 0

    # -- lifecycle --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().sph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state ------------------------------------------------------------------
    def ghosts_body(self, b: int = 0) -> np.ndarray:
        out = np.zeros((self.n_ghost[b], 2))
        check(lib().sph_ghosts_body(self._h, b, out.ctypes.data_as(C.POINTER(C.c_double))), "sph_ghosts_body")
        return out

    def state(self, stream=None):
        """(xv [N, 4] float32, body [B, 6] float64) device tensors."""
        xv = torch.empty((self.n_total, 4), dtype=torch.float32, device="cuda")
        body = torch.empty((self.B, 6), dtype=torch.float64, device="cuda")
        check(lib().sph_get_state(self._h, _ptr(xv), _ptr(body), _stream(stream)), "sph_get_state")
        return xv, body

    def set_state(self, xv, body, stream=None):
        xv = _dev(xv, torch.float32).reshape(self.n_total, 4)
        body = _dev(body, torch.float64).reshape(self.B, 6)
        check(lib().sph_set_state(self._h, _ptr(xv), _ptr(body), _stream(stream)), "sph_set_state")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    # -- stepping -------------------------------------------------------------
    def samples_for(self, n_steps: int) -> int:
        ns = C.c_int32()
        check(lib().sph_samples_for(self._h, n_steps, C.byref(ns)), "sph_samples_for")
        return ns.value

    def step(self, n_steps: int, u=None, ctrl: dict | None = None, theta_ref=None, record: bool = True,
             y_out=None, stream=None):
        """Advance n_steps; u: [B, n_steps, 3] (or [n_steps, 3] for B = 1).
        Returns the samples [B, n_samples, 11] (device) or None."""
        if u is not None:
            u = _dev(u, torch.float64).reshape(self.B, n_steps, 3)
        ref = None
        stride = 0
        if theta_ref is not None:
            ref = _dev(theta_ref, torch.float64).reshape(self.B, -1)
            stride = ref.shape[1]
            if stride < self.samples_for(n_steps):
                raise ValueError("theta_ref needs one value per sample of this call")
        c = make_ctrl(ctrl, ref, stride)
        y = y_out
        if record and y is None:
            y = torch.zeros((self.B, self.samples_for(n_steps), NY), dtype=torch.float64, device="cuda")
        check(lib().sph_step(self._h, _ptr(u), n_steps, None if c is None else C.byref(c), _ptr(y),
                             _stream(stream)), "sph_step")
        self._keep = (u, ref, y)  # keep inputs alive until the next call
        self.steps_done += n_steps
        return y

    def relax(self, n_steps: int, damping: float = 2e-3, stream=None):
        """Damped steps with the tank held fixed (relaxation of a spawned fluid)."""
        check(lib().sph_relax(self._h, n_steps, damping, _stream(stream)), "sph_relax")
        self.steps_done += n_steps

    def jvp(self, K: int, u=None, du=None, dxv0=None, dbody0=None, stream=None):
        """Forward-mode derivative of K steps along the trajectory they compute.
        Returns (y, dy, dxv, dbody): primal samples [B, n, 11], their tangent,
        and the tangent of the final fluid [N, 4] and body [B, 6] state."""
        u = None if u is None else _dev(u, torch.float64).reshape(self.B, K, 3)
        du = None if du is None else _dev(du, torch.float64).reshape(self.B, K, 3)
        dxv0 = None if dxv0 is None else _dev(dxv0, torch.float32).reshape(self.n_total, 4)
        dbody0 = None if dbody0 is None else _dev(dbody0, torch.float64).reshape(self.B, 6)
        ns = self.samples_for(K)
        y = torch.zeros((self.B, ns, NY), dtype=torch.float64, device="cuda")
        dy = torch.zeros_like(y)
        dxv = torch.empty((self.n_total, 4), dtype=torch.float32, device="cuda")
        dbody = torch.empty((self.B, 6), dtype=torch.float64, device="cuda")
        check(lib().sph_jvp(self._h, _ptr(u), _ptr(du), _ptr(dxv0), _ptr(dbody0), K, _ptr(y), _ptr(dy), _ptr(dxv),
                            _ptr(dbody), _stream(stream)), "sph_jvp")
        self.steps_done += K
        return y, dy, dxv, dbody

    def vjp(self, K: int, u=None, ybar=None, xvbar=None, bodybar=None, checkpoint_every: int = 10, stream=None):
        """Reverse-mode derivative of K steps from the current state (sph_vjp).
        ybar: adjoint of the samples [B, n, 11]; xvbar [N, 4], bodybar [B, 6]:
        adjoints of the final state.  Returns (xvbar0 [N, 4], bodybar0 [B, 6],
        ubar [B, K, 3]) and leaves the simulator at state K."""
        u = None if u is None else _dev(u, torch.float64).reshape(self.B, K, 3)
        ns = self.samples_for(K)
        ybar = None if ybar is None else _dev(ybar, torch.float64).reshape(self.B, ns, NY)
        xvbar = None if xvbar is None else _dev(xvbar, torch.float32).reshape(self.n_total, 4)
        bodybar = None if bodybar is None else _dev(bodybar, torch.float64).reshape(self.B, 6)
        xb0 = torch.empty((self.n_total, 4), dtype=torch.float32, device="cuda")
        bb0 = torch.empty((self.B, 6), dtype=torch.float64, device="cuda")
        ub = torch.empty((self.B, K, 3), dtype=torch.float64, device="cuda")
        check(lib().sph_vjp(self._h, _ptr(u), K, _ptr(ybar), _ptr(xvbar), _ptr(bodybar), _ptr(xb0), _ptr(bb0),
                            _ptr(ub), checkpoint_every, _stream(stream)), "sph_vjp")
        self.steps_done += K
        return xb0, bb0, ub

    def eval(self, u=None, stream=None):
        """Algorithm 1 on the current state without stepping."""
        N = self.n_total
        out = {
            "rho": torch.empty(N, dtype=torch.float32, device="cuda"),
            "drho": torch.empty(N, dtype=torch.float32, device="cuda"),
            "acc": torch.empty((N, 2), dtype=torch.float32, device="cuda"),
            "nbr": torch.empty((N, 3), dtype=torch.int32, device="cuda"),
            "keys": torch.empty(N, dtype=torch.int32, device="cuda"),
            "body": torch.empty((self.B, 6), dtype=torch.float64, device="cuda"),
        }
        if u is not None:
            u = _dev(u, torch.float64).reshape(self.B, 3)
        check(lib().sph_eval(self._h, _ptr(u), _ptr(out["rho"]), _ptr(out["drho"]), _ptr(out["acc"]),
                             _ptr(out["nbr"]), _ptr(out["keys"]), _ptr(out["body"]), _stream(stream)), "sph_eval")
        return out

    def eval_jvp(self, dxv=None, dbody=None, u=None, du=None, stream=None):
        """Jacobian-vector product of the continuous dynamics at the current
        state (sph_eval_jvp): tangents of the fluid accelerations [N, 2] and
        of the body's (F_x, F_y, T_b, rddot_x, rddot_y, thetaddot) [B, 6]."""
        dxv = None if dxv is None else _dev(dxv, torch.float32).reshape(self.n_total, 4)
        dbody = None if dbody is None else _dev(dbody, torch.float64).reshape(self.B, 6)
        u = None if u is None else _dev(u, torch.float64).reshape(self.B, 3)
        du = None if du is None else _dev(du, torch.float64).reshape(self.B, 3)
        dacc = torch.empty((self.n_total, 2), dtype=torch.float32, device="cuda")
        dba = torch.empty((self.B, 6), dtype=torch.float64, device="cuda")
        check(lib().sph_eval_jvp(self._h, _ptr(u), _ptr(du), _ptr(dxv), _ptr(dbody), _ptr(dacc), _ptr(dba),
                                 _stream(stream)), "sph_eval_jvp")
        return dacc, dba

    # -- diagnostics --------------------------------------------------------------
    def check(self, reset: bool = False, raise_on_error: bool = True, stream=None) -> int:
        f = C.c_int32()
        rc = lib().sph_check(self._h, C.byref(f), int(reset), _stream(stream))
        if rc != 0 and raise_on_error:
            check(rc, "sph_check")
        return f.value

    def pair_count(self, stream=None) -> int:
        n = C.c_int64()
        check(lib().sph_pair_count(self._h, C.byref(n), _stream(stream)), "sph_pair_count")
        return n.value

    def grid_info(self, b: int = 0):
        cell = C.c_double()
        W = C.c_double()
        G = C.c_int32()
        anc = (C.c_double * 2)()
        check(lib().sph_grid_info(self._h, b, C.byref(cell), C.byref(W), C.byref(G), anc), "sph_grid_info")
        return cell.value, W.value, G.value, (anc[0], anc[1])

    def time_kernels(self, n_steps: int, stream=None):
        """Mean device time (us) of the density, force and body-update
        kernels over n_steps zero-input steps, measured with CUDA events on
        the stream."""
        us = (C.c_double * 3)()
        check(lib().sph_time_kernels(self._h, n_steps, us, _stream(stream)), "sph_time_kernels")
        self.steps_done += n_steps
        return {"density": us[0], "force": us[1], "body": us[2]}

    def set_tile(self, code: int):
        check(lib().sph_set_tile(self._h, code), "sph_set_tile")

    def autotune(self, steps: int = 20, stream=None):
        chosen = C.c_int32()
        us = (C.c_double * _lib.TILE_COUNT)()
        check(lib().sph_autotune(self._h, steps, C.byref(chosen), us, _stream(stream)), "sph_autotune")
        return chosen.value, list(us)


def run_batch(params: Sequence[dict], u_profiles, T: int, ctrl: dict | None = None, theta_ref=None, stream=None):
    """One-shot batched generation of D_N (Eq. 2): returns (y [B, n_samples, 11]
    device tensor, fluid counts [B])."""
    B = len(params)
    arr = (SphParams * B)(*[make_params(d) for d in params])
    u = _dev(u_profiles, torch.float64).reshape(B, T, 3) if u_profiles is not None else None
    oe = params[0]["outer_every"]
    ns = (T + oe - 1) // oe
    y = torch.zeros((B, ns, NY), dtype=torch.float64, device="cuda")
    ref = None if theta_ref is None else _dev(theta_ref, torch.float64).reshape(B, -1)
    c = make_ctrl(ctrl, ref, 0 if ref is None else ref.shape[1])
    npart = (C.c_int32 * B)()
    check(lib().sph_run_batch(arr, B, _ptr(u), T, None if c is None else C.byref(c), _ptr(y), npart,
                              _stream(stream)), "sph_run_batch")
    return y, list(npart)


def gamma1_estimate(params: dict) -> float:
    """Eq. 15's boundary correcting factor for a representative wall of the
    tank ``params`` (the library's ``sph_gamma1_estimate``; host-side, no
    device work)."""
    g = C.c_double()
    check(lib().sph_gamma1_estimate(C.byref(make_params(params)), C.byref(g)), "sph_gamma1_estimate")
    return g.value

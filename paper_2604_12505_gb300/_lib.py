"""ctypes loader of the in-tree CUDA library (``_lib/libgb300sloshing.so``).

There is no fallback: if the library is missing or CUDA is unavailable the
import of a simulator object raises.  Build it with
``python -m paper_2604_12505_gb300.build`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgb300sloshing.so")
_lock = threading.Lock()
_lib = None

SPH_OK = 0
ERRORS = {
    -1: "SPH_E_INVAL",
    -2: "SPH_E_NOMEM",
    -3: "SPH_E_CUDA",
    -4: "SPH_E_DIVERGED",
    -5: "SPH_E_TIMEOUT",
    -6: "SPH_E_UNSUPPORTED",
}
FLAG_NAN, FLAG_ESCAPED, FLAG_CELL_FULL, FLAG_STAGE_FULL, FLAG_TIMEOUT = 1, 2, 4, 8, 16
CELL_CAPACITY = 32
NY = 11
TILE_COUNT = 5


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SphParams(C.Structure):
    _fields_ = [
        ("R", C.c_double), ("fill", C.c_double), ("dx", C.c_double), ("h_over_dx", C.c_double),
        ("rho0", C.c_double), ("k", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
        ("gamma1", C.c_double), ("eps", C.c_double), ("m_body", C.c_double), ("J_body", C.c_double),
        ("dt", C.c_double), ("grav_x", C.c_double), ("grav_y", C.c_double), ("sigma_cubic", C.c_double),
        ("ghost_pressure_sign", C.c_double), ("n_rings", C.c_int32), ("outer_every", C.c_int32),
        ("ghost_spacing", C.c_double), ("ghost_pressure_clamp", C.c_int32),
    ]


class SphCtrl(C.Structure):
    _fields_ = [
        ("J", C.c_double), ("omega", C.c_double), ("xi", C.c_double), ("theta_ref", C.c_void_p),
        ("ref_stride", C.c_int32), ("enabled", C.c_int32),
    ]


def _declare(L):
    vp, i32, i64, dp, ip = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    P = C.POINTER(SphParams)
    sig = {
        "sph_last_error": ([], C.c_char_p),
        "sph_create": ([P, vp, C.POINTER(vp)], C.c_int),
        "sph_create_batch": ([P, i32, vp, C.POINTER(vp)], C.c_int),
        "sph_destroy": ([vp], C.c_int),
        "sph_counts": ([vp, ip, ip, ip], C.c_int),
        "sph_ghosts_body": ([vp, i32, dp], C.c_int),
        "sph_get_state": ([vp, vp, vp, vp], C.c_int),
        "sph_set_state": ([vp, vp, vp, vp], C.c_int),
        "sph_step": ([vp, vp, i32, C.POINTER(SphCtrl), vp, vp], C.c_int),
        "sph_samples_for": ([vp, i32, ip], C.c_int),
        "sph_eval": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "sph_grid_info": ([vp, i32, dp, dp, ip, dp], C.c_int),
        "sph_check": ([vp, ip, i32, vp], C.c_int),
        "sph_pair_count": ([vp, C.POINTER(i64), vp], C.c_int),
        "sph_set_tile": ([vp, i32], C.c_int),
        "sph_autotune": ([vp, i32, ip, dp, vp], C.c_int),
        "sph_relax": ([vp, i32, C.c_double, vp], C.c_int),
        "sph_jvp": ([vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp], C.c_int),
        "sph_eval_jvp": ([vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "sph_vjp": ([vp, vp, i32, vp, vp, vp, vp, vp, vp, i32, vp], C.c_int),
        "sph_time_kernels": ([vp, i32, dp, vp], C.c_int),
        "sph_run_batch": ([P, i32, vp, i32, C.POINTER(SphCtrl), vp, ip, vp], C.c_int),
        "sph_gamma1_estimate": ([P, dp], C.c_int),
        "sph_density_noalloc": ([P, vp, i32, vp, i32, dp, vp, vp], C.c_int),
        "slpv_n_params": ([i32, ip], C.c_int),
        "slpv_create": ([vp, C.POINTER(vp)], C.c_int),
        "slpv_destroy": ([vp], C.c_int),
        "slpv_set_params": ([vp, vp, vp], C.c_int),
        "slpv_get_params": ([vp, vp, vp], C.c_int),
        "slpv_normalize": ([vp, vp, vp, i32, i32, vp], C.c_int),
        "slpv_loss_grad": ([vp, vp, vp, i32, i32, i32, vp, vp, vp], C.c_int),
        "slpv_train": ([vp, vp, vp, i32, i32, i32, C.c_float, i32, vp, vp], C.c_int),
        "slpv_lbfgs": ([vp, vp, vp, i32, i32, i32, i32, vp, vp], C.c_int),
        "slpv_init_ls": ([vp, vp, vp, i32, i32, vp], C.c_int),
        "slpv_predict": ([vp, vp, i32, i32, C.c_double, vp, vp, vp], C.c_int),
        "slpv_simulate": ([vp, i32, i32, vp, vp, vp, C.c_double, C.c_double, C.c_double, C.c_double, vp, vp],
                          C.c_int),
        "lpv_create": ([vp, C.POINTER(vp)], C.c_int),
        "lpv_destroy": ([vp], C.c_int),
        "lpv_set_params": ([vp, vp, vp], C.c_int),
        "lpv_get_params": ([vp, vp, vp], C.c_int),
        "lpv_normalize": ([vp, vp, vp, vp, i32, i32, vp], C.c_int),
        "lpv_init_ls": ([vp, vp, vp, i32, i32, vp, vp], C.c_int),
        "lpv_loss_grad": ([vp, vp, vp, vp, i32, i32, dp, vp, vp], C.c_int),
        "lpv_train": ([vp, vp, vp, vp, i32, i32, i32, vp, vp], C.c_int),
        "lpv_lbfgs": ([vp, vp, vp, vp, i32, i32, i32, vp, vp], C.c_int),
        "lpv_fit": ([vp, vp, vp, i32, i32, vp, C.POINTER(vp), dp, vp], C.c_int),
        "lpv_predict": ([vp, vp, vp, i32, i32, vp, vp], C.c_int),
        "lpv_simulate": ([vp, i32, vp, vp, vp, vp, i32, vp, vp, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"CUDA library not built: {LIB_PATH} is missing (run python -m paper_2604_12505_gb300.build)")
            L = C.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def check(rc: int, what: str = ""):
    if rc != SPH_OK:
        msg = lib().sph_last_error().decode(errors="replace")
        raise SphError(rc, f"{what}: {msg}" if what else msg)

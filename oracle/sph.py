"""ctypes wrapper of the FP64 CPU oracle in ``sph_oracle.c``.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, the smoke check and the CPU
baseline of ``bench.py``; never by the product path.  It imports nothing from
the CUDA package.  Each function names the paper passage it follows; the
readings taken where the paper is silent or garbled are listed in the header
of ``sph_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc_sph.so")
_lock = threading.Lock()
_lib = None

NY = 11  # r_x r_y theta v_x v_y omega F_x F_y T c_x c_y


class Params(C.Structure):
    """Mirror of ``orc_params`` (field order matters)."""

    _fields_ = [
        ("R", C.c_double),
        ("fill", C.c_double),
        ("dx", C.c_double),
        ("h_over_dx", C.c_double),
        ("rho0", C.c_double),
        ("k", C.c_double),
        ("alpha", C.c_double),
        ("beta", C.c_double),
        ("gamma1", C.c_double),
        ("eps", C.c_double),
        ("m_body", C.c_double),
        ("J_body", C.c_double),
        ("dt", C.c_double),
        ("grav_x", C.c_double),
        ("grav_y", C.c_double),
        ("sigma_cubic", C.c_double),
        ("ghost_pressure_sign", C.c_double),
        ("ctrl_J", C.c_double),
        ("ctrl_omega", C.c_double),
        ("ctrl_xi", C.c_double),
        ("n_rings", C.c_int32),
        ("outer_every", C.c_int32),
        ("ghost_spacing", C.c_double),
        ("ghost_pressure_clamp", C.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            fp = C.POINTER(C.c_float)
            P = C.POINTER(Params)
            L.orc_w_cubic.argtypes = [C.c_double] * 3
            L.orc_w_cubic.restype = C.c_double
            L.orc_dw_cubic.argtypes = [C.c_double] * 3
            L.orc_dw_cubic.restype = C.c_double
            L.orc_w_spiky.argtypes = [C.c_double] * 2
            L.orc_w_spiky.restype = C.c_double
            L.orc_dw_spiky.argtypes = [C.c_double] * 2
            L.orc_dw_spiky.restype = C.c_double
            L.orc_fill_chord.argtypes = [C.c_double, C.c_double]
            L.orc_fill_chord.restype = C.c_double
            L.orc_tank_counts.argtypes = [P, ip, ip]
            L.orc_tank_build.argtypes = [P, dp, dp]
            L.orc_ghost_world.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            L.orc_ghost_world.restype = None
            L.orc_eval.argtypes = [P, C.c_int, dp, dp, C.c_int, dp, dp, dp, C.c_int, dp, dp, dp, dp, dp, dp, dp]
            L.orc_shepard.argtypes = [P, C.c_int, dp, dp, dp]
            L.orc_run.argtypes = [P, C.c_int, dp, dp, C.c_int, dp, dp, dp, dp, C.c_int, C.c_int, C.c_double,
                                  C.c_int, dp, dp]
            L.orc_grid_dims.argtypes = [P, dp, dp, ip]
            L.orc_cell_keys_f32.argtypes = [P, C.c_int, fp, C.c_int, C.c_double, C.c_double, ip]
            L.orc_neighbor_counts_f32.argtypes = [P, C.c_int, fp, C.c_int, C.c_int, dp, dp, C.c_int, ip, ip, ip, ip]
            L.orc_neighbor_counts_f64.argtypes = [P, C.c_int, fp, C.c_int, C.c_int, dp, dp, C.c_int, ip, C.c_double,
                                                  ip]
            L.orc_switch_counts.argtypes = [P, C.c_int, dp, dp, C.c_int, dp, dp, ip]
            L.orc_pair_count.argtypes = [P, C.c_int, dp, C.c_int, dp, dp]
            L.orc_pair_count.restype = C.c_longlong
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def params(**kw) -> Params:
    """Build an ``orc_params`` from keyword values (missing ones are zero)."""
    p = Params()
    for name, _ in Params._fields_:
        if name in kw:
            setattr(p, name, kw[name])
    return p


def h_of(p: Params) -> float:
    return p.h_over_dx * p.dx


def mass_of(p: Params) -> float:
    return p.rho0 * p.dx * p.dx


def num_threads() -> int:
    return lib().orc_num_threads()


# --- kernels (Eqs. 22, 23) -------------------------------------------------
def w_cubic(r, h, sigma=5.0 / (14.0 * np.pi)):
    return lib().orc_w_cubic(float(r), float(h), float(sigma))


def dw_cubic(r, h, sigma=5.0 / (14.0 * np.pi)):
    return lib().orc_dw_cubic(float(r), float(h), float(sigma))


def w_spiky(r, h):
    return lib().orc_w_spiky(float(r), float(h))


def dw_spiky(r, h):
    return lib().orc_dw_spiky(float(r), float(h))


def fill_chord(R, fill):
    return lib().orc_fill_chord(float(R), float(fill))


# --- boundary correcting factor (Eq. 15, Section 3.5) ----------------------
def gamma1_estimate(p: Params, phase=None, n_phase: int = 512) -> float:
    """Eq. 15's gamma1 for the reference wall described in gamma1_terms."""
    lattice, fluid, ghost = gamma1_terms(p, phase, n_phase)
    return (lattice - fluid) / ghost


def gamma1_terms(p: Params, phase=None, n_phase: int = 512):
    """The three kernel sums of Eq. 15 (lattice, fluid, ghost; see below).

    Eq. 15 for the reference wall configuration of the boundary sketch
    (Section 3.2), precomputed as Section 3.5 describes.

    A straight wall along y = 0.  Fluid on the lattice (a dx, (b + 1/2) dx),
    b >= 0; n_rings ghost layers on the lines y = -(k + 1/2) s_g with ghosts
    at x = (c + phase) s_g (s_g the ghost spacing); the particle i sits at
    (0, dx/2) in the first fluid row.  rho_i / m_i is the kernel sum of an
    interior particle of the same lattice (the density the fluid has away
    from the wall), so Eq. 15 reads
        gamma1 = (sum_lattice W - sum_f W_i,f) / sum_g W_i,g.
    phase=None averages the ghost sum over n_phase equispaced phases in
    [0, 1): along a ring the ghosts' offset against the lattice varies.
    """
    L = lib()
    dx, h = p.dx, h_of(p)
    sg = (p.ghost_spacing if p.ghost_spacing > 0 else 1.0) * dx
    sigma = p.sigma_cubic if p.sigma_cubic > 0 else 5.0 / (14.0 * np.pi)
    n = int(np.ceil(2.0 * h / dx)) + 1
    full = fluid = 0.0
    for a in range(-n, n + 1):
        for b in range(-n, n + 1):
            w = L.orc_w_cubic(dx * float(np.hypot(a, b)), h, sigma)
            full += w
            if b >= 0:
                fluid += w
    phases = [phase] if phase is not None else [(q + 0.5) / n_phase for q in range(n_phase)]
    nc = int(np.ceil(2.0 * h / sg)) + 2
    ghost = 0.0
    for ph in phases:
        for k in range(p.n_rings):
            yk = -(k + 0.5) * sg - 0.5 * dx
            for c in range(-nc, nc + 1):
                ghost += L.orc_w_cubic(float(np.hypot((c + ph) * sg, yk)), h, sigma)
    ghost /= len(phases)
    return full, fluid, ghost


# --- tank (reading R9) -----------------------------------------------------
def tank_counts(p: Params):
    nf = C.c_int32()
    ng = C.c_int32()
    if lib().orc_tank_counts(C.byref(p), C.byref(nf), C.byref(ng)):
        raise ValueError("invalid tank parameters")
    return nf.value, ng.value


def tank(p: Params):
    """Fluid positions [nf, 2] and body-frame ghost positions [ng, 2]."""
    nf, ng = tank_counts(p)
    xf = np.zeros((nf, 2))
    gB = np.zeros((max(ng, 1), 2))
    lib().orc_tank_build(C.byref(p), _d(xf), _d(gB))
    return xf, gB[:ng].copy()


def ghost_world(gB, body):
    """Eq. 21: world positions, velocities and lever arms R(theta) r_g^B."""
    gB = np.ascontiguousarray(gB, dtype=np.float64)
    body = np.ascontiguousarray(body, dtype=np.float64)
    ng = gB.shape[0]
    gw = np.zeros((ng, 2))
    gv = np.zeros((ng, 2))
    arm = np.zeros((ng, 2))
    lib().orc_ghost_world(ng, _d(gB), _d(body), _d(gw), _d(gv), _d(arm))
    return gw, gv, arm


# --- Algorithm 1 -----------------------------------------------------------
def evaluate(p: Params, x, v, gB, body, u=(0.0, 0.0, 0.0), brute=False):
    """One evaluation of Algorithm 1.  Returns a dict with rho, P, acc, drho,
    fb = [F_x, F_y, T] and body_acc."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    body = np.ascontiguousarray(body, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    nf = x.shape[0]
    ng = gB.shape[0]
    rho = np.zeros(nf)
    P = np.zeros(nf)
    acc = np.zeros((nf, 2))
    drho = np.zeros(nf)
    fb = np.zeros(3)
    ba = np.zeros(3)
    fa = np.zeros(6)
    rc = lib().orc_eval(C.byref(p), nf, _d(x), _d(v), ng, _d(gB), _d(body), _d(u), int(brute), _d(rho), _d(P),
                        _d(acc), _d(drho), _d(fb), _d(ba), _d(fa))
    if rc:
        raise MemoryError("oracle evaluation failed")
    # fb_abs: [sum |f_x|, sum |f_y|, sum |arm x f|] over the fluid-ghost pair
    # forces; fb_drho: the same for rho_i df/drho_i (see orc_eval)
    return {"rho": rho, "P": P, "acc": acc, "drho": drho, "fb": fb, "body_acc": ba, "fb_abs": fa[:3],
            "fb_drho": fa[3:]}


def shepard(p: Params, x, rho):
    x = np.ascontiguousarray(x, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    S = np.zeros(x.shape[0])
    lib().orc_shepard(C.byref(p), x.shape[0], _d(x), _d(rho), _d(S))
    return S


def run(p: Params, x, v, gB, body, n_steps, u=None, theta_ref=None, use_ctrl=False, damping=0.0, brute=False,
        record=True, fb_hist=False):
    """Runs ``n_steps`` symplectic-Euler steps (Section 3.4) from copies of the
    given state.  Returns (x, v, body, y, fb_hist)."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    body = np.array(body, dtype=np.float64, copy=True)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    u_arr = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(n_steps, 3)
    ref = None if theta_ref is None else np.ascontiguousarray(theta_ref, dtype=np.float64)
    outer = max(p.outer_every, 1)
    y = np.zeros(((n_steps + outer - 1) // outer, NY)) if record else None
    fh = np.zeros((n_steps, 3)) if fb_hist else None
    rc = lib().orc_run(C.byref(p), x.shape[0], _d(x), _d(v), gB.shape[0], _d(gB), _d(body), _d(u_arr), _d(ref),
                       int(use_ctrl), int(n_steps), float(damping), int(brute), _d(y), _d(fh))
    if rc:
        raise MemoryError("oracle run failed")
    return x, v, body, y, fh


# --- integer decisions in FP32 --------------------------------------------
def grid_dims(p: Params):
    s = C.c_double()
    W = C.c_double()
    G = C.c_int32()
    lib().orc_grid_dims(C.byref(p), C.byref(s), C.byref(W), C.byref(G))
    return s.value, W.value, G.value


def cell_keys_f32(p: Params, xy_f32, anchor):
    """Cell keys in the kernels' FP32 convention (see orc_cell_keys_f32): a
    restatement of the precision the GPU takes this integer decision in, not
    a definition of the method; cell_keys_f64 is the definition it must agree
    with away from cell boundaries."""
    xy = np.ascontiguousarray(xy_f32, dtype=np.float32)
    stride = xy.shape[1]
    keys = np.zeros(xy.shape[0], dtype=np.int32)
    lib().orc_cell_keys_f32(C.byref(p), xy.shape[0], _f(xy), stride, float(anchor[0]), float(anchor[1]), _i(keys))
    return keys


def neighbor_counts_f32(p: Params, xy_f32, gB, body, query=None):
    """FP32 neighbour counts (n_ff, n_fg2, n_fg1) of the particles in
    ``query`` (indices; all if None), brute force over all particles.  This
    restates the kernels' FP32 predicate (their convention for the integer
    decision); the definition it must agree with, except on pairs within the
    band around the support, is neighbor_counts_f64."""
    xy = np.ascontiguousarray(xy_f32, dtype=np.float32)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    body = np.ascontiguousarray(body, dtype=np.float64)
    q = None if query is None else np.ascontiguousarray(query, dtype=np.int32)
    n = xy.shape[0] if q is None else q.shape[0]
    nff = np.zeros(n, dtype=np.int32)
    nfg2 = np.zeros(n, dtype=np.int32)
    nfg1 = np.zeros(n, dtype=np.int32)
    lib().orc_neighbor_counts_f32(C.byref(p), xy.shape[0], _f(xy), xy.shape[1], gB.shape[0], _d(gB), _d(body), n,
                                  None if q is None else _i(q), _i(nff), _i(nfg2), _i(nfg1))
    return nff, nfg2, nfg1


def cell_keys_f64(p: Params, xy_f32, anchor):
    """Cell keys by their exact definition: floor((x - (anchor - W)) / s)
    in FP64 on the FP32 positions, clamped to the grid; also returns, per
    particle, whether a coordinate lies within 2^-20 s of a cell boundary
    (where the FP32 convention may take the other cell)."""
    s_, W, G = grid_dims(p)
    xy = np.asarray(xy_f32, dtype=np.float32)[:, :2].astype(np.float64)
    t = (xy - (np.asarray(anchor, dtype=np.float64) - W)) / s_
    c = np.clip(np.floor(t), 0, G - 1).astype(np.int64)
    near = np.any(np.abs(t - np.round(t)) <= 2.0 ** -20 * np.maximum(np.abs(t), 1.0), axis=1)
    return (c[:, 1] * G + c[:, 0]).astype(np.int32), near


def neighbor_counts_f64(p: Params, xy_f32, gB, body, query=None, band=2.0 ** -20):
    """Neighbour counts with the exact predicate, r^2 < (2h)^2 in FP64 on the
    FP32 positions: returns (n_ff, n_fg2, n_fg1) and their band counts (pairs
    with |r^2 - s^2| <= band s^2), each an int array over ``query``."""
    xy = np.ascontiguousarray(xy_f32, dtype=np.float32)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    body = np.ascontiguousarray(body, dtype=np.float64)
    q = None if query is None else np.ascontiguousarray(query, dtype=np.int32)
    n = xy.shape[0] if q is None else q.shape[0]
    out = np.zeros((n, 6), dtype=np.int32)
    lib().orc_neighbor_counts_f64(C.byref(p), xy.shape[0], _f(xy), xy.shape[1], gB.shape[0], _d(gB), _d(body), n,
                                  None if q is None else _i(q), float(band), _i(out))
    return (out[:, 0], out[:, 2], out[:, 4]), (out[:, 1], out[:, 3], out[:, 5])


def switch_counts(p: Params, x, v, gB, body):
    """Per particle [n_ff(2h), n_fg(2h), n_fg(h), approaching n_fg(h)]: the
    discrete switches of Algorithm 1 (see orc_switch_counts)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    body = np.ascontiguousarray(body, dtype=np.float64)
    out = np.zeros((x.shape[0], 4), dtype=np.int32)
    if lib().orc_switch_counts(C.byref(p), x.shape[0], _d(x), _d(v), gB.shape[0], _d(gB), _d(body), _i(out)):
        raise MemoryError("oracle switch counts failed")
    return out


def switches_cross(p: Params, gB, states, us):
    """Where the trajectories started from ``states`` (a list of (x, v, body)
    triples, e.g. the two ends of a central difference) under the inputs
    ``us`` (one [K, 3] array per state) take a discrete switch of Algorithm 1
    differently, over the K steps.  Returns a dict: 'support' the number of
    (step, particle) cases whose neighbour counts differ (a pair crossed the
    support of Eq. 22 or 23, where the kernels vanish with two continuous
    derivatives), 'clip' the cases whose count of approaching ghost pairs
    differs (a pair crossed the kink of Eq. 18's min(., 0)), and 'first' the
    first step of either (-1: none)."""
    cur = [(np.array(a, dtype=np.float64), np.array(b, dtype=np.float64), np.array(c, dtype=np.float64))
           for a, b, c in states]
    out = {"support": 0, "clip": 0, "first": -1}
    K = len(us[0])
    for k in range(K):
        counts = [switch_counts(p, a, b, gB, c) for a, b, c in cur]
        for c in counts[1:]:
            ns = int(np.any(c[:, :3] != counts[0][:, :3], axis=1).sum())
            nc = int((c[:, 3] != counts[0][:, 3]).sum())
            out["support"] += ns
            out["clip"] += nc
            if (ns or nc) and out["first"] < 0:
                out["first"] = k
        cur = [run(p, a, b, gB, c, 1, u=u[k:k + 1], record=False)[:3] for (a, b, c), u in zip(cur, us)]
    return out


def pair_count(p: Params, x, gB, body) -> int:
    """Fluid pairs r < 2h (ordered, j != i) plus fluid-ghost pairs r < h."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    gB = np.ascontiguousarray(gB, dtype=np.float64).reshape(-1, 2)
    body = np.ascontiguousarray(body, dtype=np.float64)
    return int(lib().orc_pair_count(C.byref(p), x.shape[0], _d(x), gB.shape[0], _d(gB), _d(body)))

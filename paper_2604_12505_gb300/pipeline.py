"""Data set generation with the batched simulator and surrogate evaluation.

Tanks           a batch of independent tanks relaxed once (Section 5.1: the
                fluid is spawned, then evolved without actuation until it is
                at rest); its rest state is kept so that several manoeuvres
                start from it.  ``run`` applies inputs held over each sampling
                period (open loop, or under the PD attitude law of Eq. 28).
dataset         the data set D_N of Eq. 2 from several launches of a batch.
sequential_rate the same tanks stepped one at a time through the single-tank
                path, for the batched-versus-sequential comparison.
nrmse           1 - BFR / 100 per channel (BFR: footnote in Section 5.3.2).

Surrogate channels: input u = [F_x, F_y, tau] applied to the body; output
y = [F_x, F_y, T] (the fluid loads on the body, Eq. 20) and the distance of
the fluid centre of mass from the tank centre minus its value at rest;
scheduling p = [fill fraction, body angular rate].
"""
from __future__ import annotations

import time

import numpy as np
import torch

from .sph import Sim


class Tanks:
    """B tanks (list of parameter dicts with one dt and outer_every) relaxed
    with ``relax_steps`` damped steps; velocities are zeroed afterwards."""

    def __init__(self, params: list[dict], relax_steps: int, damping: float = 4e-3, autotune: bool = True):
        self.params = params
        self.outer = params[0]["outer_every"]
        self.sim = Sim(params)
        if autotune:
            self.sim.autotune(steps=10)
        if relax_steps > 0:
            self.sim.relax(relax_steps, damping=damping)
        xv, body = self.sim.state()
        xv[:, 2:] = 0.0
        self.rest = (xv.clone(), body.clone())
        self.sim.set_state(*self.rest)
        self.sim.check()
        self.fill = np.array([p["fill"] for p in params])
        self.n_fluid = list(self.sim.n_fluid)

    def run(self, u_samples: np.ndarray, ctrl: dict | None = None, theta_ref: np.ndarray | None = None):
        """u_samples [B, K, 3] per sampling period, from the rest state.
        Returns (samples [B, K, 11] float64 numpy, device seconds)."""
        B, K, _ = u_samples.shape
        self.sim.set_state(*self.rest)
        u_inner = torch.tensor(np.repeat(u_samples, self.outer, axis=1), dtype=torch.float64, device="cuda")
        ref = None if theta_ref is None else torch.tensor(theta_ref, dtype=torch.float64, device="cuda")
        y = torch.zeros((B, K, 11), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        self.sim.step(K * self.outer, u=u_inner, ctrl=ctrl, theta_ref=ref, y_out=y)
        e1.record()
        torch.cuda.synchronize()
        self.sim.check()
        return y.cpu().numpy(), e0.elapsed_time(e1) * 1e-3

    def rest_of(self, b: int):
        """Rest state (xv, body) of tank b alone."""
        o = int(np.sum(self.n_fluid[:b]))
        return self.rest[0][o:o + self.n_fluid[b]].clone(), self.rest[1][b:b + 1].clone()

    def close(self):
        self.sim.close()


def surrogate_channels(y_raw: np.ndarray, fill: np.ndarray):
    """(y [B, K, 4], p [B, K, 2]) from the simulator samples [B, K, 11]."""
    off = np.linalg.norm(y_raw[:, :, 9:11] - y_raw[:, :, 0:2], axis=2)
    y = np.concatenate([y_raw[:, :, 6:9], (off - off[:, :1])[:, :, None]], axis=2)
    p = np.stack([np.broadcast_to(fill[:, None], off.shape), y_raw[:, :, 5]], axis=2)
    return y, p


def dataset(tanks: Tanks, u_launches: list[np.ndarray]):
    """D_N from one launch of the batch per input array [B, K, 3]: returns
    dict(u, y, p [L*B, K, .], tank [L*B], seconds, steps) with trajectories
    ordered launch-major."""
    us, ys, ps, secs = [], [], [], 0.0
    for u in u_launches:
        y_raw, s = tanks.run(u)
        y, p = surrogate_channels(y_raw, tanks.fill)
        us.append(u)
        ys.append(y)
        ps.append(p)
        secs += s
    B = len(tanks.params)
    K = u_launches[0].shape[1]
    return dict(u=np.concatenate(us), y=np.concatenate(ys), p=np.concatenate(ps),
                tank=np.tile(np.arange(B), len(u_launches)), seconds=secs, steps=len(u_launches) * K * tanks.outer)


def sequential_rate(tanks: Tanks, which: list[int], n_steps: int):
    """Device seconds per step of each listed tank run alone through the
    single-tank path (same tile autotuning, same rest state)."""
    out = []
    for b in which:
        s = Sim(tanks.params[b])
        s.autotune(steps=10)
        s.set_state(*tanks.rest_of(b))
        s.step(32, record=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(n_steps, record=False)
        e1.record()
        torch.cuda.synchronize()
        s.check()
        out.append(e0.elapsed_time(e1) * 1e-3 / n_steps)
        s.close()
    return out


def nrmse(y: np.ndarray, yh: np.ndarray) -> np.ndarray:
    """1 - BFR / 100 per channel, BFR = 1 - ||y - yh|| / ||y - mean(y)||."""
    num = np.sqrt(np.sum((y - yh) ** 2, axis=0))
    den = np.sqrt(np.sum((y - y.mean(axis=0)) ** 2, axis=0))
    return num / np.maximum(den, 1e-300)


def _closed_loop_inputs(B: int, K: int, Ts: float, seed0: int):
    """Held-out manoeuvres: F and tau from the data-set distribution, theta_ref random steps."""
    from . import workloads as W

    F = np.stack([W.piecewise_profile(K, Ts, seed=seed0 + b)[:, :2] for b in range(B)])
    tau = np.stack([W.piecewise_profile(K, Ts, seed=seed0 + 10_000 + b)[:, 2] for b in range(B)])
    ref = np.stack([W.theta_ref_steps(K, Ts, seed=seed0 + 20_000 + b) for b in range(B)])
    return F, tau, ref


def identification_inputs(B: int, K: int, Ts: float, seed0: int) -> np.ndarray:
    """[B, K, 3] identification trains (Section 5.3.1), one per tank, with the
    paper's design scaled from its 2200 samples of 0.05 s (110 s) to a horizon
    of K samples of Ts: the multisine keeps its 39 lines with the resolution
    of one period over its segment (the paper's 0.05 Hz over 82.5 s), and the
    pulse widths and rests shrink by the same factor."""
    from . import workloads as W

    horizon = K * Ts
    scale = horizon / (2200 * 0.05)
    f_res = 1.0 / (0.75 * horizon)
    return np.stack([W.identification_train(K, Ts, seed=seed0 + b, f_res=f_res, f_max=40 * f_res,
                                            pulse_width=(0.25 * scale, 1.0 * scale),
                                            pulse_rest=(1.0 * scale, 4.0 * scale)) for b in range(B)])


def scheduling_use(model, u, y, p, train) -> dict:
    """Whether a fitted LPV model (Eq. 24, p = [fill, thetadot]) uses its
    scheduling: the Frobenius norm of each M_i (i >= 1) and of its A, B and C
    blocks relative to M_0's, and the held-out open-loop output NRMSE of the
    model as fitted, with p frozen at its training mean, and with one
    channel of p frozen at a time."""
    W = model.get_params()[0].astype(np.float64)
    c = model.cfg
    nx = c["n_x"]
    blocks = dict(A=(slice(0, nx), slice(0, nx)), B=(slice(0, nx), slice(nx, None)),
                  C=(slice(nx, None), slice(0, nx)))
    rel = lambda a, b: float(np.linalg.norm(a) / max(np.linalg.norm(b), 1e-300))
    norms = {f"M{i}": dict(all=rel(W[i], W[0]), **{k: rel(W[i][r, q], W[0][r, q]) for k, (r, q) in blocks.items()})
             for i in range(1, W.shape[0])}
    pt, pm = p[~train][:, :, :c["n_p"]], p[train][:, :, :c["n_p"]].reshape(-1, c["n_p"]).mean(axis=0)
    yt, ut = y[~train], u[~train]

    def held_out(pp):
        yh = model.predict(ut, pp).cpu().numpy()
        return np.mean([nrmse(a, b) for a, b in zip(yt, yh)], axis=0).tolist()

    frozen = dict(fitted=held_out(pt), all_frozen=held_out(np.broadcast_to(pm, pt.shape).copy()))
    for j, name in enumerate(["fill", "thetadot"][:c["n_p"]]):
        q = pt.copy()
        q[:, :, j] = pm[j]
        frozen[f"{name}_frozen"] = held_out(q)
    return dict(weight_norm_vs_M0=norms, p_train_mean=pm.tolist(), held_out_output_nrmse=frozen)


def surrogate_study(n_tanks: int = 256, launches: int = 4, steps: int = 10_000, relax: int = 5000,
                    dt: float = 2e-4, cl_tanks: int = 64, cl_steps: int = 5000, n_sims: int = 65_536,
                    fit_cfg: dict | None = None, seq_tanks: int | None = None, seq_steps: int = 200, ctrl=None,
                    log=None, inputs: str = "piecewise", fill=(0.2, 0.8), dx=(0.004, 0.01)) -> dict:
    """The surrogate workflow on the simulator and the LPV library.

    1. D_N: n_tanks tanks (fill ~ U[fill], dx ~ U[dx]: a degenerate range
       such as dx=(0.006, 0.006) gives tanks that differ only in fill) relaxed
       once, ``launches`` open-loop runs of ``steps`` steps each with seeded
       inputs -- piecewise-constant holds (``inputs="piecewise"``) or the
       identification train scaled to the horizon (``inputs="train"``); the
       batch step rate against the same tanks stepped one at a time (every
       tank, ``seq_steps`` steps each, unless ``seq_tanks`` limits them).
    2. Fit (lpv.fit) on the trajectories of the first 80 % of the tanks, for
       the LPV model (p = [fill, thetadot]) and the LTI model (no scheduling).
    3. cl_tanks unseen tanks under unseen manoeuvres in closed loop with the PD
       attitude law (Eq. 28) for cl_steps steps, by the simulator and by the
       surrogate; NRMSE per body channel, and throughput of n_sims surrogate
       closed-loop runs against the simulator's.
    """
    from . import lpv
    from . import workloads as W

    say = log or (lambda *a: None)
    ctrl = ctrl or dict(omega=0.2 * np.pi, xi=0.7)
    out: dict = {}
    params = [dict(p, dt=dt) for p in W.batch_tank_params(n_tanks, seed0=1000, fill=fill, dx=dx)]
    outer = params[0]["outer_every"]
    Ts = dt * outer
    K = steps // outer
    t0 = time.perf_counter()
    tanks = Tanks(params, relax)
    out["relax_wall_s"] = time.perf_counter() - t0
    if inputs == "piecewise":
        u_l = [np.stack([W.piecewise_profile(K, Ts, seed=100_000 + 1000 * l + b) for b in range(n_tanks)])
               for l in range(launches)]
    elif inputs == "train":
        u_l = [identification_inputs(n_tanks, K, Ts, seed0=100_000 + 1000 * l) for l in range(launches)]
    else:
        raise ValueError(f"inputs must be 'piecewise' or 'train', not {inputs!r}")
    out["inputs"] = inputs
    d = dataset(tanks, u_l)
    npart = np.array(tanks.n_fluid, dtype=np.float64)
    n_seq = n_tanks if seq_tanks is None else min(seq_tanks, n_tanks)
    seq = sequential_rate(tanks, list(range(n_seq)), seq_steps)
    s_batch = d["seconds"] / d["steps"]
    if n_seq == n_tanks:   # every tank timed alone: the sequential step is their sum
        s_seq = float(np.sum(seq))
        how = f"all {n_tanks} tanks alone, {seq_steps} steps each, summed"
    else:
        s_seq = float(np.sum(seq) / npart[:len(seq)].sum() * npart.sum())
        how = f"{len(seq)} of {n_tanks} tanks alone, {seq_steps} steps each, scaled to all tanks by particle count"
    out["dataset"] = dict(trajectories=int(d["u"].shape[0]), samples=K, tanks=n_tanks, particles=int(npart.sum()),
                          device_s=d["seconds"], batched_ms_per_step=1e3 * s_batch,
                          sequential_ms_per_step=1e3 * s_seq, batched_speedup=s_seq / s_batch,
                          sequential_sample=how)
    say("dataset", out["dataset"])
    tanks.close()

    ntr = int(round(0.8 * n_tanks))
    tr = d["tank"] < ntr
    cfg = dict(lpv.DEFAULT, **(fit_cfg or {}))
    u, y, p = d["u"], d["y"], d["p"]
    fits = {}
    for name, n_p in (("lpv", 2), ("lti", 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model, best = lpv.fit(u[tr], y[tr], p[tr][:, :, :n_p], dict(cfg, n_p=n_p))
        torch.cuda.synchronize()
        fit_s = time.perf_counter() - t0
        yh = model.predict(u[~tr], p[~tr][:, :, :n_p]).cpu().numpy()
        e = np.mean([nrmse(a, b) for a, b in zip(y[~tr], yh)], axis=0)
        fits[name] = model
        out[f"fit_{name}"] = dict(train_loss=best, seconds=fit_s, test_nrmse_outputs=e.tolist())
        say("fit", name, out[f"fit_{name}"])
    out["scheduling"] = scheduling_use(fits["lpv"], u, y, p, tr)
    say("scheduling", out["scheduling"])

    pt = [dict(q, dt=dt) for q in W.batch_tank_params(cl_tanks, seed0=2000, fill=fill, dx=dx)]
    Kc = cl_steps // outer
    F, tau, ref = _closed_loop_inputs(cl_tanks, Kc, Ts, seed0=200_000)
    tt = Tanks(pt, relax)
    ys, sph_s = tt.run(np.concatenate([F, tau[:, :, None]], axis=2), ctrl=ctrl, theta_ref=ref)
    ys = ys[:, :, :6]
    fill = tt.fill
    tt.close()
    body = dict(m=pt[0]["m_body"], J=pt[0]["J_body"], Ts=Ts, n_sub=outer, ctrl_omega=ctrl["omega"],
                ctrl_xi=ctrl["xi"])
    names = ["r_x", "r_y", "theta", "rdot_x", "rdot_y", "thetadot"]

    def cl_err(model):
        yl = model.simulate(F, tau, ref, fill, body).cpu().numpy()
        e = np.mean([nrmse(ys[b], yl[b]) for b in range(cl_tanks)], axis=0)
        return dict(zip(names, e.tolist())), float(np.mean(e[[2, 5]])), float(np.mean(e[[0, 1, 3, 4]]))

    none = lpv.Model(dict(fits["lpv"].cfg))
    none.set_params(np.zeros(none.shape_W, dtype=np.float32), fits["lpv"].get_params()[1])
    lti = lpv.Model(dict(fits["lpv"].cfg))
    Wl = np.zeros(lti.shape_W, dtype=np.float32)
    W0, s0 = fits["lti"].get_params()
    Wl[0] = W0[0]
    lti.set_params(Wl, np.concatenate([s0, fits["lpv"].get_params()[1][len(s0):]]))
    for name, m in (("lpv", fits["lpv"]), ("lti", lti), ("no_fluid", none)):
        per, att, trn = cl_err(m)
        out[f"closed_loop_{name}"] = dict(nrmse=per, nrmse_attitude=att, nrmse_translation=trn,
                                          nrmse_mean=float(np.mean(list(per.values()))),
                                          all_channels_within_5pct=bool(max(per.values()) <= 0.05))
        say("closed loop", name, out[f"closed_loop_{name}"])

    # throughput: n_sims surrogate runs (the held-out manoeuvres tiled), inputs resident
    idx = np.arange(n_sims) % cl_tanks
    dev = lambda a: torch.tensor(a[idx], dtype=torch.float64, device="cuda")
    Fd, td, rd, fd = dev(F), dev(tau), dev(ref), dev(fill)
    model = fits["lpv"]
    model.simulate(Fd[:256], td[:256], rd[:256], fd[:256], body)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    model.simulate(Fd, td, rd, fd, body)
    e1.record()
    torch.cuda.synchronize()
    lpv_s = e0.elapsed_time(e1) * 1e-3
    out["throughput"] = dict(surrogate_sims=n_sims, surrogate_s=lpv_s, surrogate_sims_per_s=n_sims / lpv_s,
                             sph_sims=cl_tanks, sph_s=sph_s, sph_sims_per_s=cl_tanks / sph_s,
                             speedup=(n_sims / lpv_s) / (cl_tanks / sph_s), steps=cl_steps, periods=Kc, Ts=Ts, dt=dt)
    say("throughput", out["throughput"])
    return out


def size_sweep(dxs=(0.02, 0.005, 0.002, 0.0014, 0.001, 0.0007), relax: int = 3000, steps: int = 1000,
               log=None) -> list:
    """Step time against tank size: the R = 0.5 m, 50 % fill tank at each dx
    (dt = 5e-5 s), relaxed with `relax` damped steps, autotuned, then `steps`
    graph-replayed steps timed with CUDA events; plus the Tables 1-2
    spacecraft with three rings.  Reports particles, tile, us per step, pair
    interactions per step and per second, and the health flags."""
    from . import workloads as W

    say = log or (lambda *a: None)
    cases = [(f"R=0.5 m, dx={dx}", dict(W.BASE, dx=dx)) for dx in dxs] + [("Tables 1-2, three rings", dict(W.PAPER_RINGS))]
    out = []
    for name, cfg in cases:
        with Sim(cfg) as sim:
            sim.relax(relax, damping=2e-3)
            xv, body = sim.state()
            xv[:, 2:] = 0.0
            sim.set_state(xv, body)
            tile, _ = sim.autotune(steps=32)
            sim.step(64, record=False)
            c0 = sim.pair_count()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.step(steps, record=False)
            e1.record()
            torch.cuda.synchronize()
            us = 1e3 * e0.elapsed_time(e1) / steps
            pairs = (sim.pair_count() - c0) / steps
            r = dict(tank=name, particles=int(sim.n_fluid[0]), tile=int(tile), us_per_step=us, pairs_per_step=pairs,
                     pairs_per_s=pairs / (us * 1e-6), flags=sim.check(reset=True, raise_on_error=False))
        say("size sweep", r)
        out.append(r)
    return out


def linearization_study(cfg: dict | None = None, relax: int = 2000, steps: int = 2000, n_points: int = 3,
                        tau: float = 5.0, block: int = 1024, log=None) -> dict:
    """Eigenvalues of the linearised dynamics along a manoeuvre (Section 5.2,
    the Jacobian of xdot = f(x, u) by automatic differentiation): the tank
    (by default the paper's benchmark spacecraft) relaxed to rest, then a
    torque slew (+tau, then -tau) of ``steps`` steps; A = df/dx at n_points
    evenly spaced steps from the library's Jacobian-vector products, and its
    spectrum.  Reports the timings and, per point, the spectral abscissa
    (largest real part), the spectral radius and the number of eigenvalues
    with real part above 1e-6 of the radius."""
    from . import autodiff as AD
    from . import workloads as W
    from .sph import Sim

    say = log or (lambda *a: None)
    cfg = dict(cfg or W.PAPER_RINGS)
    with Sim(cfg) as sim:
        sim.relax(relax, damping=2e-3)
        xv, body = sim.state()
        xv[:, 2:] = 0.0
        n_f = xv.shape[0]
    u = W.bang_bang_slew(steps, cfg["dt"], tau=tau, t1=steps * cfg["dt"] / 2)
    at = np.linspace(0, steps, n_points).round().astype(int)
    out = dict(particles=n_f, n=4 * n_f + 6, steps=steps, dt=cfg["dt"], points=[])
    with Sim(cfg) as sim:
        sim.set_state(xv, body[0])
        k = 0
        for ka in at:
            if ka > k:
                sim.step(int(ka - k), u=torch.tensor(u[k:ka], device="cuda")[None], record=False)
                k = int(ka)
            x, b = sim.state()
            sim.check()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = AD.jacobian(cfg, x, b[0], u[ka] if ka < steps else None, block=block)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ev = torch.linalg.eigvals(A.cpu())  # host LAPACK (a dense nonsymmetric eigensolver)
            t2 = time.perf_counter()
            re, mag = ev.real, ev.abs()
            rad = mag.max().item()
            pt = dict(step=int(ka), t=float(ka * cfg["dt"]), jacobian_s=t1 - t0, eig_s=t2 - t1,
                      abscissa=re.max().item(), radius=rad, n_unstable=int((re > 1e-6 * rad).sum().item()),
                      theta=float(b[0, 2].item()))
            out["points"].append(pt)
            say("linearization", pt)
    return out


def paper_scenario_study(seconds: float = 30.0, relax: int = 20_000, batch: int = 64, jitter: float = 0.25,
                         seed: int = 0, gammas=None, extra: dict | None = None, log=None) -> dict:
    """The paper's benchmark spacecraft (Section 5.1, Tables 1 and 2) on this
    GPU, as context for the simulation times the paper reports (Table 3).

    Spawn: the 6 mm lattice with each coordinate moved by U(-jitter, jitter) dx
    (seeded), then relaxed with the tank held fixed (damping 2e-3 per step):
    Section 5.1 spawns the particles at random and lets them come to rest.
    Flight: `seconds` at dt = 1 ms with seeded piecewise forces and torques,
    the PD attitude law of Eq. 28 sampled every 50 ms tracking random attitude
    steps.  Run with Table 2's wall (one layer of 0.9 dx ghosts) for each
    gamma1 in `gammas` (default: Table 2's 0.5, Eq. 15's estimate from
    ``sph_gamma1_estimate``, and 1.5), and with this repository's wall (three
    rings at dx, gamma1 = 1.5), each on one tank (the wall time of one
    sph_step call over the whole flight, and the largest fluid radius over R
    checked every second, against the outermost ghost ring) and on `batch`
    copies with their own spawns and inputs stepped together.  The health flags (SPH_FLAG_*)
    after the relaxation and after each flight are recorded; a gamma1 whose
    relaxation already lets fluid through the wall is not flown.  `extra`
    (e.g. dict(ghost_pressure_clamp=1): Eq. 16 with max(P_i, 0)) is applied to Table 2's
    walls."""
    from . import workloads as W
    from .sph import Sim, gamma1_estimate

    say = log or (lambda *a: None)
    base = dict(W.PAPER, **(extra or {}))
    outer, dt = base["outer_every"], base["dt"]
    Ts = outer * dt
    K = int(round(seconds / Ts))
    g15 = gamma1_estimate(base)
    walls = [dict(base, gamma1=g) for g in gammas] if gammas is not None else \
        [base, dict(base, gamma1=g15), dict(base, gamma1=1.5), dict(W.PAPER_RINGS)]
    F, tau, ref = _closed_loop_inputs(batch, K, Ts, seed0=3000 + seed)
    u = np.concatenate([F, tau[..., None]], axis=2)                       # [batch, K, 3]
    ctrl = dict(omega=base["ctrl_omega"], xi=base["ctrl_xi"])
    out = dict(seconds=seconds, steps=K * outer, dt=dt, Ts=Ts, gamma1_eq15=g15, jitter_dx=jitter,
               paper=dict(profile1_s=9.9093, horizon_s=30.0, hardware="RTX 2000 Ada laptop GPU, JAX (Table 3)"),
               runs=[])

    def spawn(sim, seeds):
        xv, body = sim.state()
        x = xv.cpu().numpy()
        o = 0
        for b, n in enumerate(sim.n_fluid):
            x[o:o + n, :2] += W.uniform_jitter((n, 2), jitter * base["dx"], seed=seeds[b])
            o += n
        sim.set_state(x, body)
        sim.relax(relax, damping=2e-3)
        flags = sim.check(reset=True, raise_on_error=False)
        xv, body = sim.state()
        vmax = float(xv[:, 2:].norm(dim=1).max().item())
        xv[:, 2:] = 0.0
        sim.set_state(xv, body)
        return vmax, flags

    for cfg in walls:
        run = dict(gamma1=cfg["gamma1"], rings=cfg["n_rings"], ghost_spacing=cfg["ghost_spacing"],
                   ghost_pressure_clamp=cfg.get("ghost_pressure_clamp", 0))
        with Sim(cfg) as sim:
            run["particles"], run["ghosts"] = sim.n_fluid[0], sim.n_ghost[0]
            run["relax_vmax"], run["relax_flags"] = spawn(sim, [seed])
            if run["relax_flags"]:
                say("paper scenario", run)
                out["runs"].append(run)
                continue
            rest = sim.state()
            ui = torch.tensor(np.repeat(u[:1], outer, axis=1), dtype=torch.float64, device="cuda")
            rf = torch.tensor(ref[:1], dtype=torch.float64, device="cuda")
            sim.step(10 * outer, u=ui[:, :10 * outer], ctrl=ctrl, theta_ref=rf[:, :10], record=False)  # warm-up
            sim.set_state(*rest)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0 = time.perf_counter()
            e0.record()
            sim.step(K * outer, u=ui, ctrl=ctrl, theta_ref=rf)
            e1.record()
            torch.cuda.synchronize()
            run["one_tank_wall_s"] = time.perf_counter() - w0
            run["one_tank_device_s"] = e0.elapsed_time(e1) * 1e-3
            run["flight_flags"] = sim.check(reset=True, raise_on_error=False)
            # the same flight in one-second pieces, for the largest radius
            sim.set_state(*rest)
            per = int(round(1.0 / Ts))
            rmax = 0.0
            for k0 in range(0, K, per):
                k1 = min(K, k0 + per)
                sim.step((k1 - k0) * outer, u=ui[:, k0 * outer:k1 * outer], ctrl=ctrl, theta_ref=rf[:, k0:k1],
                         record=False)
                xv, body = sim.state()
                d = xv[:, :2].double() - body[0, :2]
                rmax = max(rmax, float(d.norm(dim=1).max().item()))
            sim.check(reset=True, raise_on_error=False)
            run["max_radius_over_R"] = rmax / base["R"]
            run["escaped_past_ghosts"] = bool(rmax > base["R"] + (cfg["n_rings"] - 0.5) * cfg["ghost_spacing"] * base["dx"])
        with Sim([cfg] * batch) as sim:
            sim.autotune(steps=10)
            _, bflags = spawn(sim, [seed + 1 + b for b in range(batch)])
            ub = torch.tensor(np.repeat(u, outer, axis=1), dtype=torch.float64, device="cuda")
            rb = torch.tensor(ref, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.step(K * outer, u=ub, ctrl=ctrl, theta_ref=rb, record=False)
            e1.record()
            torch.cuda.synchronize()
            tb = e0.elapsed_time(e1) * 1e-3
            xv, body = sim.state()
            lim = base["R"] + (cfg["n_rings"] - 0.5) * cfg["ghost_spacing"] * base["dx"]
            o, past = 0, []
            for b, n in enumerate(sim.n_fluid):
                d = (xv[o:o + n, :2].double() - body[b, :2]).norm(dim=1)
                past.append(int((~(d <= lim)).sum().item()))
                o += n
            run["batch"] = dict(tanks=batch, device_s=tb, flights_per_s=batch / tb, relax_flags=bflags,
                                flight_flags=sim.check(reset=True, raise_on_error=False),
                                tanks_past_ghosts=int(sum(q > 0 for q in past)),
                                particles_past_ghosts=int(sum(past)))
        run["speedup_vs_paper_one_tank"] = out["paper"]["profile1_s"] * (seconds / 30.0) / run["one_tank_wall_s"]
        say("paper scenario", run)
        out["runs"].append(run)
    return out


def velocity_surrogate_study(n_train: int = 24, n_val: int = 8, id_samples: int = 2200, relax: int = 20_000,
                             lti_iters: int = 1000, lti_lr: float = 1e-3, adam_iters: int = 0, lr: float = 1e-4,
                             lbfgs_iters: int = 1000, m1_std: float = 0.0, restarts: int = 8, cl_samples: int = 600,
                             n_sims: int = 65_536,
                             nx: int = 4, net_scale: float = 1.0,
                             sigma2: float = 1e-4, seed: int = 0, log=None) -> dict:
    """The paper's identification study (Section 5.3) on its spacecraft.

    1. D_N: n_train copies of the Tables 1-2 spacecraft (three ghost rings,
       `workloads.PAPER_RINGS`), relaxed, each driven open loop by its own
       identification train (pulses, then a random-phase multisine on
       [0, 2) Hz at 0.05 Hz; 2200 samples at T_s = 0.05 s) and sampled every
       T_s: inputs u = [F_x, F_y, tau], outputs the body velocities
       [rdot_x, rdot_y, thetadot] (the velocity-level reformulation).
    2. The self-scheduled LPV model (n_x = 4, n_p = 1, eta a 2 x 4 tanh
       network, D = 0): an LTI stage (M_0 only: the least-squares ARX start,
       then Adam on the free-run loss) stands in for the ssest fit; then
       `restarts` LPV fits from it with M_1's B and C blocks ~ N(0, m1_std^2)
       (zero by default: the restart starts on the LTI fit, where the
       gradient of M_1 is already nonzero) and Xavier network weights:
       adam_iters Adam steps on M_1 and the network (M_0 held; none by
       default), then L-BFGS on all of theta; the lowest training loss kept.
    3. Validation as in Table 3: n_val closed-loop manoeuvres of
       cl_samples * T_s seconds (the PD law of Eq. 28 tracking random attitude
       steps, piecewise forces and torques) flown by the SPH simulator and by
       the augmented surrogates (LTI and LPV) with the same inputs; BFR per
       channel (r_x, r_y, theta, rdot_x, rdot_y, thetadot).
    4. Throughput: n_sims surrogate closed loops at once, against the
       simulator's flights per second on the validation batch."""
    from . import workloads as W
    from .slpv import VelocityModel, initial_theta

    say = log or (lambda *a: None)
    cfg = dict(W.PAPER_RINGS)
    Ts = cfg["dt"] * cfg["outer_every"]
    out = dict(Ts=Ts, id_samples=id_samples, n_train=n_train, n_val=n_val, nx=nx)
    t0 = time.perf_counter()
    tanks = Tanks([cfg] * n_train, relax_steps=relax)
    u_id = np.stack([W.identification_train(id_samples, Ts, seed=5000 + seed * 1000 + b) for b in range(n_train)])
    ys, sec = tanks.run(u_id)
    tanks.close()
    out["dataset"] = dict(sph_device_s=sec, wall_s=time.perf_counter() - t0)
    u = torch.tensor(u_id, dtype=torch.float32, device="cuda")
    y = torch.tensor(ys[:, :, 3:6], dtype=torch.float32, device="cuda")
    say("velocity surrogate: data", out["dataset"])

    m = VelocityModel(nx=nx, sigma2=sigma2)
    m.normalize(u, y)
    _, sc = m.get_params()
    t1 = time.perf_counter()
    m.init_ls(u, y)
    fits = dict(ls=dict(loss=float(m.loss_grad(u, y, grad=False)[0].item())))
    h = m.train(u, y, lti_iters, lti_lr, stage=m.LTI).cpu().numpy() if lti_iters > 0 else np.array([np.nan])
    th_lti, _ = m.get_params()
    fits["lti"] = dict(loss=float(m.loss_grad(u, y, grad=False)[0].item()), seconds=time.perf_counter() - t1)
    # the LTI fit is itself a member of the scheduled family (M_1 = 0, the
    # network at zero, where every gradient of M_1 and of the network
    # vanishes): it is the first candidate, so that the kept model fits the
    # training data at least as well as the LTI one
    best = (fits["lti"]["loss"], th_lti, -1)
    for r in range(restarts):
        t2 = time.perf_counter()
        m.set_params(initial_theta(nx, seed=seed * 100 + r + 1, base=th_lti, m1_std=m1_std, net_scale=net_scale), sc)
        l0 = float(m.loss_grad(u, y, grad=False)[0].item())
        # Adam on the scheduling part (M_0 held at the LTI fit), then L-BFGS on everything
        if adam_iters > 0:
            m.train(u, y, adam_iters, lr, stage=m.SCHEDULING)
        if lbfgs_iters > 0 and np.isfinite(float(m.loss_grad(u, y, grad=False)[0].item())):
            m.lbfgs(u, y, lbfgs_iters)
        loss = float(m.loss_grad(u, y, grad=False)[0].item())
        fits.setdefault("restart_losses", []).append([l0, loss])
        say("velocity surrogate: restart", r, l0, loss, time.perf_counter() - t2)
        if np.isfinite(loss) and loss < best[0]:
            best = (loss, m.get_params()[0], r)
    fits["lpv"] = dict(loss=best[0], seconds=time.perf_counter() - t1 - fits["lti"]["seconds"],
                       restarts=restarts, adam_iters=adam_iters, lbfgs_iters=lbfgs_iters, m1_std=m1_std,
                       kept=("the LTI fit (no restart lowered its training loss)" if best[2] < 0
                             else f"restart {best[2]}"))
    out["fit"] = fits
    # training-set BFR of the free run (velocities)
    yv = ys[:, :, 3:6]

    def bfr_of(model_theta):
        m.set_params(model_theta, sc)
        vh, _ = m.predict(u, Ts)
        vh = vh.cpu().numpy()
        return [float(100.0 * (1.0 - np.mean([nrmse(yv[b, :, c], vh[b, :, c]) for b in range(n_train)])))
                for c in range(3)]

    out["train_bfr_velocity"] = dict(lti=bfr_of(th_lti), lpv=bfr_of(best[1]) if best else None)

    # closed-loop validation (Table 3 style)
    K = cl_samples
    F, tau, ref = _closed_loop_inputs(n_val, K, Ts, seed0=7000 + seed)
    ctrl = dict(omega=cfg["ctrl_omega"], xi=cfg["ctrl_xi"])
    val = Tanks([cfg] * n_val, relax_steps=relax)
    ysph, t_sph = val.run(np.concatenate([F, tau[..., None]], axis=2), ctrl=ctrl, theta_ref=ref)
    val.close()
    ref_traj = ysph[:, :, :6]
    chans = ("r_x", "r_y", "theta", "rdot_x", "rdot_y", "thetadot")
    out["validation"] = dict(seconds=K * Ts, sph_device_s=t_sph, sph_flights_per_s=n_val / t_sph)
    for name, th in (("lti", th_lti), ("lpv", best[1] if best else th_lti)):
        m.set_params(th, sc)
        sim = m.simulate(F, tau, ref, Ts, cfg["J_body"], ctrl["omega"], ctrl["xi"]).cpu().numpy()
        bfr = {c: float(100.0 * (1.0 - np.mean([nrmse(ref_traj[b, :, i], sim[b, :, i]) for b in range(n_val)])))
               for i, c in enumerate(chans)}
        out["validation"][name] = bfr
        say("velocity surrogate: closed-loop BFR", name, bfr)
    # throughput of the surrogate closed loop
    reps = (n_sims + n_val - 1) // n_val  # the validation inputs repeated on the device
    Fb = torch.tensor(F, device="cuda").repeat(reps, 1, 1)[:n_sims].contiguous()
    tb = torch.tensor(tau, device="cuda").repeat(reps, 1)[:n_sims].contiguous()
    rb = torch.tensor(ref, device="cuda").repeat(reps, 1)[:n_sims].contiguous()
    m.simulate(Fb[:64], tb[:64], rb[:64], Ts, cfg["J_body"], ctrl["omega"], ctrl["xi"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    m.simulate(Fb, tb, rb, Ts, cfg["J_body"], ctrl["omega"], ctrl["xi"])
    e1.record()
    torch.cuda.synchronize()
    t_sur = e0.elapsed_time(e1) * 1e-3
    out["throughput"] = dict(surrogate_sims=n_sims, samples=K, surrogate_s=t_sur, surrogate_sims_per_s=n_sims / t_sur,
                             sph_flights_per_s=n_val / t_sph, speedup=(n_sims / t_sur) / (n_val / t_sph))
    m.close()
    return out


if __name__ == "__main__":
    import json
    import sys

    if len(sys.argv) > 1 and sys.argv[1] == "linearize":
        print(json.dumps(linearization_study(log=lambda *a: print(*a, file=sys.stderr))))
    elif len(sys.argv) > 1 and sys.argv[1] == "paper":
        # "paper clamp": Table 2's walls with Eq. 16 taking max(P_i, 0)
        extra = dict(ghost_pressure_clamp=1) if "clamp" in sys.argv[2:] else None
        print(json.dumps(paper_scenario_study(extra=extra, log=lambda *a: print(*a, file=sys.stderr))))
    elif len(sys.argv) > 1 and sys.argv[1] == "surrogate":
        # "surrogate fill_only": the data-set workload with every tank at dx = 6 mm
        kw = dict(fit_cfg=dict(adam_iters=2000, restarts=8, lbfgs_iters=100), seq_tanks=8)
        if "fill_only" in sys.argv[2:]:
            kw["dx"] = (0.006, 0.006)
        r = surrogate_study(**kw, log=lambda *a: print(*a, file=sys.stderr))
        print(json.dumps(r))
    elif len(sys.argv) > 1 and sys.argv[1] == "sweep":
        print(json.dumps(size_sweep(log=lambda *a: print(*a, file=sys.stderr))))
    elif len(sys.argv) > 1 and sys.argv[1] == "velocity":
        print(json.dumps(velocity_surrogate_study(log=lambda *a: print(*a, file=sys.stderr))))
    else:
        print("usage: python -m paper_2604_12505_gb300.pipeline linearize|paper [clamp]|surrogate [fill_only]|sweep|velocity",
              file=sys.stderr)
        sys.exit(2)

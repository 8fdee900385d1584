"""Parity at the benchmark's full sizes, on sampled outputs the oracle can
compute one by one: the 256-tank data-set batch (about 2.5 M particles) and
the 65,536-run surrogate closed loop; plus the one-shot batch entry point."""
import numpy as np
import pytest

from oracle import lpv as L
from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, normwise, traj_err

pytestmark = pytest.mark.gpu


def test_one_shot_batch_equals_stepping_the_batch():
    torch = need_gpu()
    from paper_2604_12505_gb300.sph import Sim, run_batch
    params = [dict(p, dx=p["dx"] * 2.0) for p in W.batch_tank_params(6, seed0=1300)]
    T = 60
    u = np.stack([W.piecewise_profile(T, params[0]["dt"], seed=90 + b, hold=(0.0005, 0.001)) for b in range(6)])
    y1, npart = run_batch(params, u, T)
    with Sim(params) as s:
        y2 = s.step(T, u=u)
        assert npart == s.n_fluid
    assert torch.equal(y1, y2)


def test_full_data_set_batch_sampled_tanks_match_oracle(orc):
    need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    params = [dict(p, dt=2e-4, outer_every=1) for p in W.batch_tank_params(256, seed0=1000)]
    n = 10
    sample = [0, 77, 255]
    u = np.stack([W.piecewise_profile(n, 2e-4, seed=300 + b, hold=(0.0004, 0.001)) for b in range(256)])
    with Sim(params) as s:
        assert sum(s.n_fluid) > 2_000_000
        xv, body = [t.cpu().numpy() for t in s.state()]
        out = s.eval()
        rho = out["rho"].cpu().numpy()
        acc = out["acc"].cpu().numpy()
        y = s.step(n, u=u).cpu().numpy()
        s.check()
        off = s.offsets
    for b in sample:
        p = orc.params(**params[b])
        _, gB = orc.tank(p)
        x64 = xv[off[b]:off[b + 1], :2].astype(np.float64)
        v64 = xv[off[b]:off[b + 1], 2:].astype(np.float64)
        ref = orc.evaluate(p, x64, v64, gB, body[b])
        assert np.abs(rho[off[b]:off[b + 1]] - ref["rho"]).max() / ref["rho"].min() <= 1e-5
        assert normwise(acc[off[b]:off[b + 1]], ref["acc"]) <= 1e-5
        yr = orc.run(p, x64, v64, gB, body[b], n, u=u[b])[3]
        err = traj_err(y[b], yr)
        assert max(err.values()) <= 1e-3, (b, err)


def test_full_closed_loop_batch_sampled_runs_match_oracle():
    need_gpu()
    from paper_2604_12505_gb300.lpv import Model
    rng = np.random.default_rng(41)
    nx = 12
    m = Model(dict(n_p=2))
    Wt = np.zeros(m.shape_W)
    for i in range(3):
        A = rng.normal(size=(nx, nx))
        A *= (0.6 if i == 0 else 0.1) / np.linalg.norm(A, 2)
        Wt[i, :nx, :nx] = A
        Wt[i, :nx, nx:] = 0.05 * rng.normal(size=(nx, 3))
        Wt[i, nx:, :nx] = 0.05 * rng.normal(size=(4, nx))
    scales = np.array([20, 20, 2, 30, 30, 3, 0.05, 0.5, 0.0, 0.2, 0.05, 0.2, -0.05, 0.8, 0.05], dtype=np.float32)
    m.set_params(Wt, scales)
    W32 = m.get_params()[0].transpose(1, 0, 2).reshape(16, -1).astype(np.float64)
    B, T = 65_536, 500
    F = rng.uniform(-20, 20, size=(B, T, 2))
    tau = rng.uniform(-2, 2, size=(B, T))
    ref = np.repeat(rng.uniform(-0.3, 0.3, size=(B, 5)), T // 5, axis=1)
    fill = rng.uniform(0.2, 0.8, size=B)
    body = dict(m=500.0, J=50.0, Ts=2e-3, n_sub=10, ctrl_omega=0.2 * np.pi, ctrl_xi=0.7)
    out = m.simulate(F, tau, ref, fill, body).cpu().numpy()
    sc = dict(u=scales[:3].astype(float), y=scales[3:7].astype(float), p_mean=scales[7:9].astype(float),
              p_scale=scales[9:11].astype(float))
    for b in (0, 12345, 65535):
        o = L.closed_loop(W32, nx, sc, body, fill[b], F[b], tau[b], ref[b], body["Ts"], body["n_sub"],
                          dict(omega=body["ctrl_omega"], xi=body["ctrl_xi"]),
                          p_range=(scales[11:13].astype(float), scales[13:15].astype(float)))
        for cols in ([0, 1], [2], [3, 4], [5]):
            den = np.linalg.norm(o[:, cols], axis=1).max()
            assert np.linalg.norm(out[b][:, cols] - o[:, cols], axis=1).max() <= 1e-3 * den, (b, cols)

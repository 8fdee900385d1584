"""GPU tests of the data-set generation and surrogate workflow
(paper_2604_12505_gb300/pipeline.py) on small batches."""
import numpy as np
import pytest

from tests.gpu_util import need_gpu


def _params(B, seed0=1000, dt=2e-4):
    from paper_2604_12505_gb300 import workloads as W
    return [dict(p, dt=dt, dx=p["dx"] * 2.0) for p in W.batch_tank_params(B, seed0=seed0)]


@pytest.mark.gpu
def test_relaxed_batch_runs_match_single_tank_runs_bit_exactly():
    need_gpu()
    from paper_2604_12505_gb300 import pipeline as PL, workloads as W
    from paper_2604_12505_gb300.sph import Sim
    import torch
    params = _params(5)
    tanks = PL.Tanks(params, relax_steps=500, autotune=False)
    K = 30
    u = np.stack([W.piecewise_profile(K, 2e-3, seed=40 + b, hold=(0.005, 0.02)) for b in range(5)])
    y, _ = tanks.run(u)
    for b in (0, 3):
        s = Sim(params[b])
        s.set_state(*tanks.rest_of(b))
        yb = s.step(K * 10, u=torch.tensor(np.repeat(u[b:b + 1], 10, axis=1), device="cuda")).cpu().numpy()
        np.testing.assert_array_equal(yb[0], y[b])
        s.close()
    # a second launch from the rest state repeats the first
    y2, _ = tanks.run(u)
    np.testing.assert_array_equal(y2, y)
    tanks.close()


def test_surrogate_channels():
    from paper_2604_12505_gb300 import pipeline as PL
    rng = np.random.default_rng(0)
    y_raw = rng.normal(size=(3, 7, 11))
    fill = np.array([0.2, 0.5, 0.8])
    y, p = PL.surrogate_channels(y_raw, fill)
    np.testing.assert_array_equal(y[:, :, :3], y_raw[:, :, 6:9])
    off = np.hypot(y_raw[:, :, 9] - y_raw[:, :, 0], y_raw[:, :, 10] - y_raw[:, :, 1])
    np.testing.assert_allclose(y[:, :, 3], off - off[:, :1], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(p[:, :, 0], np.repeat(fill[:, None], 7, axis=1))
    np.testing.assert_array_equal(p[:, :, 1], y_raw[:, :, 5])


@pytest.mark.gpu
def test_small_surrogate_study_end_to_end():
    need_gpu()
    from paper_2604_12505_gb300 import pipeline as PL
    r = PL.surrogate_study(n_tanks=10, launches=2, steps=1000, relax=1000, cl_tanks=5, cl_steps=1000, n_sims=2048,
                           fit_cfg=dict(adam_iters=20, restarts=1), seq_tanks=2, seq_steps=100)
    assert r["dataset"]["trajectories"] == 20 and r["dataset"]["samples"] == 100
    assert r["dataset"]["batched_speedup"] > 1.0
    for name in ("lpv", "lti", "no_fluid"):
        c = r[f"closed_loop_{name}"]
        assert all(np.isfinite(v) for v in c["nrmse"].values())
    th = r["throughput"]
    assert th["surrogate_sims"] == 2048 and th["periods"] == 100
    assert th["surrogate_sims_per_s"] > th["sph_sims_per_s"]


@pytest.mark.gpu
def test_study_on_the_identification_train():
    need_gpu()
    from paper_2604_12505_gb300 import pipeline as PL
    r = PL.surrogate_study(n_tanks=10, launches=1, steps=1000, relax=1000, cl_tanks=5, cl_steps=1000, n_sims=1024,
                           fit_cfg=dict(adam_iters=20, restarts=1), seq_tanks=2, seq_steps=100, inputs="train")
    assert r["inputs"] == "train" and r["dataset"]["trajectories"] == 10
    for name in ("lpv", "lti", "no_fluid"):
        assert all(np.isfinite(v) for v in r[f"closed_loop_{name}"]["nrmse"].values())


@pytest.mark.gpu
def test_paper_scenario_study_short():
    """The Tables 1-2 spacecraft: one 236-ghost layer, a jittered spawn relaxed
    to rest, a short PD-controlled flight per gamma1, health flags recorded."""
    need_gpu()
    from paper_2604_12505_gb300 import pipeline as PL
    r = PL.paper_scenario_study(seconds=1.0, relax=1000, batch=2, gammas=[0.5, 1.5])
    assert r["steps"] == 1000 and [x["gamma1"] for x in r["runs"]] == [0.5, 1.5]
    assert 0.5 < r["gamma1_eq15"] < 2.0
    for run in r["runs"]:
        assert run["particles"] == 2024 and run["ghosts"] == 236
        assert isinstance(run["relax_flags"], int) and np.isfinite(run["relax_vmax"])
        if run["relax_flags"] == 0:
            assert run["one_tank_device_s"] > 0 and 0.5 < run["max_radius_over_R"]
            assert run["batch"]["tanks"] == 2 and run["batch"]["flights_per_s"] > 0


@pytest.mark.gpu
def test_velocity_surrogate_study_short():
    """The paper's identification study at toy sizes: data from the spacecraft
    under identification trains, LTI and LPV fits, closed-loop BFR."""
    need_gpu()
    from paper_2604_12505_gb300 import pipeline as PL
    r = PL.velocity_surrogate_study(n_train=3, n_val=2, id_samples=200, relax=1000, lti_iters=30, adam_iters=30,
                                    restarts=2, cl_samples=100, n_sims=1024)
    assert r["fit"]["lti"]["loss"] > 0 and np.isfinite(r["fit"]["lpv"]["loss"])
    assert len(r["train_bfr_velocity"]["lpv"]) == 3
    for name in ("lti", "lpv"):
        assert set(r["validation"][name]) == {"r_x", "r_y", "theta", "rdot_x", "rdot_y", "thetadot"}
        assert all(np.isfinite(v) for v in r["validation"][name].values())
    assert r["throughput"]["surrogate_sims"] == 1024 and r["throughput"]["speedup"] > 1.0

"""What the scheduling of the LPV surrogate gains on simulator data
(Section 4, Eq. 24 with p = [fill, thetadot]; Section 5.3.2 fit).

Data: 128 tanks of the data-set family (R = 0.5 m, fill ~ U[0.2, 0.8],
dx ~ U[6, 10] mm, seeds 5000+), relaxed, then two open-loop launches of
10,000 SPH steps at dt = 2e-4 s under seeded piecewise forces and torques,
sampled every 2 ms (256 trajectories of 1000 samples).  The fit runs on the
trajectories of the first 80 % of the tanks; the held-out 20 % are tanks
the fit never saw.  Tile shape fixed (no autotuning), so the data are the
same on every run.

The free-run prediction of the loads F_b and T_b over 2 s is no better than
their mean for either model (NRMSE about 1): the floating fluid's wall
impacts are not linear.  The distance of the fluid's centre of mass from the
tank centre is where the scheduling pays: the body rate moves the fluid out
to the wall, an effect bilinear in the rate and the state that an LTI model
cannot represent.  Asserted:
  * the LPV model's held-out NRMSE of the centre-of-mass offset is at most
    0.85 of the LTI model's;
  * freezing thetadot at its training mean raises it by at least 1.25x: the
    gain comes from the scheduling, not from the larger model.
The fluid's wall impacts make the data sensitive to the last bits of the
arithmetic, and the fits to the data: on this family the measured ratios
ranged over 0.45-0.77 (LPV against LTI) and 1.4-2.1 (thetadot frozen) across
data sets and builds, hence the margins.
"""
import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_scheduled_model_predicts_the_fluid_offset_better_than_lti():
    need_gpu()
    from paper_2604_12505_gb300 import lpv
    from paper_2604_12505_gb300 import pipeline as P
    from paper_2604_12505_gb300 import workloads as W

    n_tanks, K, Ts = 128, 1000, 2e-3
    params = [dict(p, dt=2e-4) for p in W.batch_tank_params(n_tanks, seed0=5000, dx=(0.006, 0.01))]
    tanks = P.Tanks(params, 5000, autotune=False)
    u_l = [np.stack([W.piecewise_profile(K, Ts, seed=100_000 + 1000 * l + b) for b in range(n_tanks)])
           for l in range(2)]
    d = P.dataset(tanks, u_l)
    tanks.close()
    tr = d["tank"] < int(round(0.8 * n_tanks))
    u, y, p = d["u"], d["y"], d["p"]
    err, models = {}, {}
    for name, n_p in (("lpv", 2), ("lti", 0)):
        m, best = lpv.fit(u[tr], y[tr], p[tr][:, :, :n_p],
                          dict(lpv.DEFAULT, adam_iters=1000, restarts=4, n_p=n_p))
        assert np.isfinite(best)
        yh = m.predict(u[~tr], p[~tr][:, :, :n_p]).cpu().numpy()
        err[name] = np.mean([P.nrmse(a, b) for a, b in zip(y[~tr], yh)], axis=0)
        models[name] = m
    sched = P.scheduling_use(models["lpv"], u, y, p, tr)
    frozen = np.array(sched["held_out_output_nrmse"]["thetadot_frozen"])
    print(f"held-out NRMSE [F_x, F_y, T, CoM offset]: LPV {np.round(err['lpv'], 3)}, LTI {np.round(err['lti'], 3)}, "
          f"LPV with thetadot frozen {np.round(frozen, 3)}; |M1|/|M0| {sched['weight_norm_vs_M0']['M1']['all']:.3f}")
    assert err["lpv"][3] <= 0.85 * err["lti"][3], (err["lpv"], err["lti"])
    assert frozen[3] >= 1.25 * err["lpv"][3], (frozen, err["lpv"])

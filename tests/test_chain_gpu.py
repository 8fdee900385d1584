"""Steps launched as a chain equal steps launched one call at a time, bit for
bit.

Inside a run of steps (a captured graph of 32 steps, the steps after it, a
relaxation), the density pass of every step after the first stages its tile
and sums the fluid part of Eq. 14 before its grid dependency on the previous
step's body update, reading what the previous force pass wrote.  A step
launched by a call of its own waits first.  Both orders of work take the
same arithmetic, so any read of data not yet written would show as a
difference: 40 steps in one call (a graph of 32, then 8 chained steps) must
equal 40 calls of one step, in the samples, the state and the body, on the
938-particle tank and on the 97,748-particle benchmark tank (1024 tiles, two
waves of CTAs per pass)."""
import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W
from tests.gpu_util import need_gpu, oracle_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg, tile", [(W.SMALL, 3), (W.LARGE, 4)])
def test_chained_steps_equal_single_step_calls(orc, cfg, tile):
    torch = need_gpu()
    from paper_2604_12505_gb300.sph import Sim
    xv, *_ = oracle_state(orc, cfg, 0.2, 0.05, seed=21)
    n = 40
    u = W.bang_bang_slew(n, cfg["dt"], tau=50.0, t1=n * cfg["dt"] / 2)
    body0 = np.array([0.001, -0.002, 0.1, 0.01, 0.02, 0.5])
    with Sim(cfg) as s:
        s.set_tile(tile)
        s.set_state(xv, body0)
        ya = s.step(n, u=u[None]).cpu().numpy()
        xa, ba = [t.cpu().numpy() for t in s.state()]
        s.check()
        s.set_state(xv, body0)
        yb = np.concatenate([s.step(1, u=u[None, k:k + 1]).cpu().numpy() for k in range(n)], axis=1)
        xb, bb = [t.cpu().numpy() for t in s.state()]
        s.check()
        # and a relaxation (chained) against single damped steps
        s.set_state(xv, body0)
        s.relax(n, damping=1e-3)
        xr, br = [t.cpu().numpy() for t in s.state()]
        s.set_state(xv, body0)
        for _ in range(n):
            s.relax(1, damping=1e-3)
        xs, bs = [t.cpu().numpy() for t in s.state()]
        s.check()
    np.testing.assert_array_equal(ya, yb)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ba, bb)
    np.testing.assert_array_equal(xr, xs)
    np.testing.assert_array_equal(br, bs)

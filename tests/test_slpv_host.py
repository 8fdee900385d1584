"""Host-side pieces of the self-scheduled surrogate front end (no GPU): the
parameter layout agrees with the oracle's, and the starting points of a fit
have the structure of Section 5.3.2: a random LTI start (A_0 = 0.9 I, M_1
and the network at zero), and restarts that keep M_0, draw M_1's B and C
blocks (its A and D blocks zero) and Xavier network weights with zero
biases."""
import numpy as np
import pytest

from oracle import slpv as S


@pytest.mark.parametrize("nx", [2, 4, 6, 8])
def test_layout_matches_the_oracle(nx):
    from paper_2604_12505_gb300.slpv import layout
    L = layout(nx)
    sizes = [L[k].stop - L[k].start for k in ("M0", "M1", "W1", "b1", "W2", "b2", "w3", "b3")]
    assert sizes == S.sizes(nx, 3, 3)
    assert L["b3"].stop == 2 * (nx + 3) ** 2 + 4 * (nx + 3) + 29


def test_starting_points():
    from paper_2604_12505_gb300.slpv import initial_theta, layout
    nx = 4
    L = layout(nx)
    lti = initial_theta(nx, seed=1)
    P = S.unpack(lti.astype(np.float64), nx, 3, 3)
    np.testing.assert_array_equal(P["M0"][:nx, :nx], 0.9 * np.eye(nx).astype(np.float32))
    assert np.all(P["M0"][nx:, nx:] == 0) and np.all(lti[L["M0"].stop:] == 0)
    lpv = initial_theta(nx, seed=2, base=lti, m1_std=0.01)
    Q = S.unpack(lpv.astype(np.float64), nx, 3, 3)
    np.testing.assert_array_equal(lpv[L["M0"]], lti[L["M0"]])          # M_0 kept
    assert np.all(Q["M1"][:nx, :nx] == 0) and np.all(Q["M1"][nx:, nx:] == 0)  # A and D blocks of M_1 zero
    assert np.abs(Q["M1"]).max() > 0
    for name, fan_in, fan_out in (("W1", nx + 3, 4), ("W2", 4, 4), ("w3", 4, 1)):
        assert np.abs(Q[name]).max() <= np.sqrt(6.0 / (fan_in + fan_out)) + 1e-7   # Xavier's uniform bound
    assert np.all(Q["b1"] == 0) and np.all(Q["b2"] == 0) and np.all(Q["b3"] == 0)
    on_lti = initial_theta(nx, seed=3, base=lti, m1_std=0.0)
    assert np.all(on_lti[L["M1"]] == 0)                                  # a restart on the LTI fit
    np.testing.assert_array_equal(initial_theta(nx, seed=2, base=lti, m1_std=0.01), lpv)  # seeded

"""Pins of the oracle's ghost layers (Section 3.2, Table 2) and of its Eq. 15
estimate of the boundary correcting factor gamma1 (Section 3.5), checked
against values the paper prints and against closed forms."""
import os

import numpy as np
import pytest

from paper_2604_12505_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_ghost_count.txt")


def _golden():
    row = [ln for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")][0].split()
    return float(row[0]), float(row[1]), float(row[2]), int(row[3])


def test_table2_single_ghost_layer(orc):
    """One ring of 5.4 mm ghosts around the 0.2 m tank holds Table 2's 236."""
    R, dx, ds, n_printed = _golden()
    p = orc.params(**dict(W.PAPER, R=R, dx=dx, ghost_spacing=ds / dx, n_rings=1))
    assert orc.tank_counts(p)[1] == n_printed
    _, gB = orc.tank(p)
    r = np.hypot(gB[:, 0], gB[:, 1])
    np.testing.assert_allclose(r, R + 0.5 * ds, rtol=0, atol=1e-15)  # a layer one ghost thick outside the wall
    ang = np.sort(np.arctan2(gB[:, 1], gB[:, 0]))
    gaps = np.diff(np.r_[ang, ang[:1] + 2 * np.pi]) * r[0]
    assert np.abs(gaps - ds).max() <= 1e-3 * ds  # equispaced at the ghost length


def test_ghost_spacing_default_is_the_lattice_spacing(orc):
    a = orc.tank(orc.params(**W.SMALL))[1]
    b = orc.tank(orc.params(**dict(W.SMALL, ghost_spacing=1.0)))[1]
    np.testing.assert_array_equal(a, b)
    assert orc.tank_counts(orc.params(**W.SMALL)) == (938, 500)


@pytest.mark.parametrize("h_over_dx", [1.3, 9.42 / 6.0, 2.0])
def test_gamma1_is_one_when_ghosts_complete_the_lattice(orc, h_over_dx):
    """Ghost rows at the lattice spacing and phase, deep enough to fill the
    support, are exactly the particles missing beyond the wall (Eq. 13 with no
    missing term), so Eq. 15 must return 1."""
    n_rows = int(np.ceil(2 * h_over_dx)) + 1
    p = orc.params(**dict(W.SMALL, h_over_dx=h_over_dx, n_rings=n_rows, ghost_spacing=1.0))
    assert abs(orc.gamma1_estimate(p, phase=0.0) - 1.0) <= 1e-13
    # the same rows shifted half a spacing along the wall are not the lattice
    assert abs(orc.gamma1_estimate(p, phase=0.5) - 1.0) > 1e-6


@pytest.mark.parametrize("cfg", [dict(W.PAPER, n_rings=1, ghost_spacing=0.9),
                                 dict(W.SMALL, n_rings=3, ghost_spacing=1.0),
                                 dict(W.SMALL, n_rings=2, ghost_spacing=1.2)])
def test_phase_averaged_ghost_sum_is_the_line_integral(orc, cfg):
    """Averaged over the offset along the wall, a row of ghosts spaced s_g
    sums to (1/s_g) times the integral of W along the row (Poisson summation)."""
    integrate = pytest.importorskip("scipy.integrate")
    p = orc.params(**cfg)
    h, dx = orc.h_of(p), p.dx
    sg = p.ghost_spacing * dx
    ref = 0.0
    for k in range(p.n_rings):
        d = 0.5 * dx + (k + 0.5) * sg
        if d >= 2 * h:
            continue
        xm = np.sqrt(4 * h * h - d * d)
        pts = [np.sqrt(h * h - d * d)] if d < h else None
        val, _ = integrate.quad(lambda x: orc.w_cubic(np.hypot(x, d), h), -xm, xm, points=pts,
                                epsabs=0, epsrel=1e-12, limit=200)
        ref += val / sg
    ghost = orc.gamma1_terms(p, n_phase=2048)[2]
    assert abs(ghost - ref) <= 1e-8 * ref


def test_gamma1_falls_as_ghost_rows_are_added(orc):
    g = [orc.gamma1_estimate(orc.params(**dict(W.SMALL, n_rings=n))) for n in (1, 2, 3, 4)]
    assert g[0] > g[1]
    # seen from the first fluid row (dx/2 inside the wall) the third ghost row
    # lies 3 dx away, beyond the support 2h = 2.6 dx: it changes nothing
    assert g[3] == g[2] == g[1]


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_ghost_pressure_clamp_reading(orc, sign):
    # With ghost_pressure_clamp = 1 Eq. 16 takes max(P_i, 0).  A
    # lone particle next to one ghost has rho_i = m (W(0) + gamma1 W(r)), far
    # below rho0, so P_i < 0: as printed (clamp 0) the wall term pulls it
    # towards the ghost for the repulsive sign (-1); clamped, the wall exerts
    # no pressure force at all, and at P_i > 0 the clamp changes nothing.
    base = dict(W.BASE, dx=0.01, beta=0.0, ghost_pressure_sign=sign)
    gB = np.array([[0.2, 0.0]])
    h = orc.h_of(orc.params(**base))
    x = np.array([[0.2 - 0.6 * h, 0.0]])
    v = np.zeros((1, 2))
    free = orc.evaluate(orc.params(**base), x, v, gB, np.zeros(6))
    clamped = orc.evaluate(orc.params(**dict(base, ghost_pressure_clamp=1)), x, v, gB, np.zeros(6))
    assert free["P"][0] < 0
    towards = (gB[0] - x[0]) @ free["acc"][0]
    assert (towards > 0) if sign < 0 else (towards < 0)
    np.testing.assert_array_equal(clamped["acc"], 0.0)
    np.testing.assert_array_equal(clamped["fb"], 0.0)
    # a heavy ghost weight compresses the particle (rho_i / rho0 = dx^2 (W(0) +
    # gamma1 W(r)) is 3.6 at gamma1 = 20): P_i > 0, and the clamp is the identity
    hi = dict(base, gamma1=20.0)
    a = orc.evaluate(orc.params(**hi), x, v, gB, np.zeros(6))
    b = orc.evaluate(orc.params(**dict(hi, ghost_pressure_clamp=1)), x, v, gB, np.zeros(6))
    assert a["P"][0] > 0
    np.testing.assert_array_equal(a["acc"], b["acc"])

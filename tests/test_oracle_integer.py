"""Pins of the oracle's FP32 integer decisions (cell keys and neighbour
counts), the decisions the GPU kernels must reproduce bit for bit."""
import numpy as np

from paper_2604_12505_gb300 import workloads as W


def test_cell_stencil_covers_support(orc):
    # Every pair closer than 2h lies in neighbouring cells (|dcol|, |drow| <= 1),
    # so a 3x3 stencil finds every neighbour.
    p = orc.params(**W.SMALL)
    x, gB = orc.tank(p)
    x = (x + W.perturbation(x.shape, 0.3 * p.dx, seed=11)).astype(np.float32)
    s, Wd, G = orc.grid_dims(p)
    assert s > 2 * orc.h_of(p)
    anchor = (0.0123, -0.0071)
    keys = orc.cell_keys_f32(p, x, anchor)
    col, row = keys % G, keys // G
    xd = x.astype(np.float64)
    d2 = ((xd[:, None, :] - xd[None, :, :]) ** 2).sum(-1)
    i, j = np.nonzero(d2 < (2 * orc.h_of(p)) ** 2)
    assert np.all(np.abs(col[i] - col[j]) <= 1)
    assert np.all(np.abs(row[i] - row[j]) <= 1)
    # and the key is the floor of the scaled offset (away from cell edges)
    t = (xd - (np.array(anchor) - Wd)) / s
    ok = np.abs(t - np.round(t)).min(axis=1) > 1e-4
    np.testing.assert_array_equal(col[ok], np.floor(t[ok, 0]).astype(int))
    np.testing.assert_array_equal(row[ok], np.floor(t[ok, 1]).astype(int))


def test_fp32_neighbour_counts_agree_with_exact_distances(orc):
    # The FP32 predicate agrees with the exact distance test except for pairs
    # whose squared distance sits within FP32 rounding of the support.
    p = orc.params(**W.TINY)
    x, gB = orc.tank(p)
    x = (x + W.perturbation(x.shape, 0.3 * p.dx, seed=12)).astype(np.float32)
    body = np.array([0.001, 0.002, 0.3, 0.0, 0.0, 0.0])
    nff, nfg2, nfg1 = orc.neighbor_counts_f32(p, x, gB, body)
    h = orc.h_of(p)
    xd = x.astype(np.float64)
    d2 = ((xd[:, None, :] - xd[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    exact = (d2 < (2 * h) ** 2).sum(1)
    near = (np.abs(d2 - (2 * h) ** 2) < 1e-5 * (2 * h) ** 2).sum(1)
    assert np.all(np.abs(nff - exact) <= near)
    gw, _, _ = orc.ghost_world(gB, body)
    dg = ((xd[:, None, :] - gw[None, :, :]) ** 2).sum(-1)
    assert np.all(np.abs(nfg2 - (dg < (2 * h) ** 2).sum(1)) <= (np.abs(dg - 4 * h * h) < 4e-5 * h * h).sum(1))
    assert np.all(np.abs(nfg1 - (dg < h * h).sum(1)) <= (np.abs(dg - h * h) < 1e-5 * h * h).sum(1))
    assert nff.sum() > 10 * len(x) and nfg1.sum() > 0


def test_pair_count_equals_fp32_counts_away_from_the_support(orc):
    p = orc.params(**W.TINY)
    x, gB = orc.tank(p)
    body = np.array([0.0, 0.0, 0.2, 0.0, 0.0, 0.0])
    x = x + W.perturbation(x.shape, 0.2 * p.dx, seed=13)
    nff, _, nfg1 = orc.neighbor_counts_f32(p, x.astype(np.float32), gB, body)
    x32 = x.astype(np.float32).astype(np.float64)
    assert orc.pair_count(p, x32, gB, body) == int(nff.sum() + nfg1.sum())


def test_fp64_predicate_counts_equal_brute_force(orc):
    # The exact predicate: r^2 < (2h)^2 (r^2 < h^2 for Eqs. 16-18) in FP64
    # on the FP32 positions, against an independent NumPy brute force.
    p = orc.params(**W.TINY)
    x, gB = orc.tank(p)
    x = (x + W.perturbation(x.shape, 0.3 * p.dx, seed=14)).astype(np.float32)
    body = np.array([0.002, -0.001, 0.7, 0.0, 0.0, 0.0])
    (nff, nfg2, nfg1), (bff, bfg2, bfg1) = orc.neighbor_counts_f64(p, x, gB, body)
    h = orc.h_of(p)
    xd = x.astype(np.float64)
    d2 = ((xd[:, None, :] - xd[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    np.testing.assert_array_equal(nff, (d2 < (2 * h) ** 2).sum(1))
    np.testing.assert_array_equal(bff, (np.abs(d2 - (2 * h) ** 2) <= 2.0 ** -20 * (2 * h) ** 2).sum(1))
    c, s = np.cos(body[2]), np.sin(body[2])
    gw = body[:2] + gB @ np.array([[c, s], [-s, c]])  # R(theta) r_g^B + r, written out
    dg = ((xd[:, None, :] - gw[None, :, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(nfg2, (dg < (2 * h) ** 2).sum(1))
    np.testing.assert_array_equal(nfg1, (dg < h * h).sum(1))
    assert nfg1.sum() > 0 and nff.sum() > 10 * len(x)


def test_fp32_convention_agrees_with_the_fp64_definition_up_to_the_band(orc):
    # The kernels' FP32 predicate (restated by neighbor_counts_f32) may decide
    # only the pairs inside the band around the support differently.  A
    # lattice puts many pairs exactly at the lattice spacings, some of which
    # fall near 2h for h = 1.3 dx only after the jitter.
    for cfg, seed in ((W.TINY, 15), (W.SMALL, 16)):
        p = orc.params(**cfg)
        x, gB = orc.tank(p)
        x = (x + W.perturbation(x.shape, 0.25 * p.dx, seed=seed)).astype(np.float32)
        body = np.array([0.003, 0.001, -0.4, 0.0, 0.0, 0.0])
        f32 = orc.neighbor_counts_f32(p, x, gB, body)
        f64, band = orc.neighbor_counts_f64(p, x, gB, body)
        for a, b, w in zip(f32, f64, band):
            assert np.all(np.abs(a - b) <= w)


def test_fp32_cell_keys_agree_with_the_fp64_definition_off_the_boundaries(orc):
    p = orc.params(**W.SMALL)
    x, gB = orc.tank(p)
    x = (x + W.perturbation(x.shape, 0.3 * p.dx, seed=17)).astype(np.float32)
    anchor = (0.0311, -0.0177)
    k32 = orc.cell_keys_f32(p, x, anchor)
    k64, near = orc.cell_keys_f64(p, x, anchor)
    np.testing.assert_array_equal(k32[~near], k64[~near])
    assert near.sum() < len(x) // 100


def test_switch_counts_and_crossing_detector(orc):
    # Two particles straddling the support 2h by +-1e-9 relative: the
    # detector reports a support crossing at the first step; a particle
    # moving towards a ghost within h counts as approaching, one moving away
    # does not, and the detector sees that clip cross.
    p = orc.params(**dict(W.BASE, dx=0.01))
    h = orc.h_of(p)
    far = np.zeros((0, 2))
    body = np.array([50.0, 50.0, 0.0, 0.0, 0.0, 0.0])
    pair = lambda d: np.array([[0.0, 0.0], [d, 0.0]])
    v0 = np.zeros((2, 2))
    assert orc.switch_counts(p, pair(2 * h * (1 - 1e-9)), v0, far, body)[:, 0].tolist() == [1, 1]
    assert orc.switch_counts(p, pair(2 * h * (1 + 1e-9)), v0, far, body)[:, 0].tolist() == [0, 0]
    u = np.zeros((3, 3))
    r = orc.switches_cross(p, far, [(pair(2 * h * (1 - 1e-9)), v0, body), (pair(2 * h * (1 + 1e-9)), v0, body)], [u, u])
    assert r["support"] == 2 * 3 and r["clip"] == 0 and r["first"] == 0   # both particles, each of the 3 steps
    gB = np.array([[0.2, 0.0]])
    b0 = np.zeros(6)
    x = np.array([[0.2 - 0.5 * h, 0.0]])
    towards, away = np.array([[1e-3, 0.0]]), np.array([[-1e-3, 0.0]])
    assert orc.switch_counts(p, x, towards, gB, b0)[0].tolist()[2:] == [1, 1]
    assert orc.switch_counts(p, x, away, gB, b0)[0].tolist()[2:] == [1, 0]
    r = orc.switches_cross(p, gB, [(x, towards, b0), (x, away, b0)], [u[:1], u[:1]])
    assert r["clip"] == 1 and r["first"] == 0
    # a generic tiny perturbation of a resting lattice crosses nothing in a few steps
    q = orc.params(**W.TINY)
    xt, gt = orc.tank(q)
    xt = xt + W.perturbation(xt.shape, 0.2 * q.dx, seed=18)
    e = 1e-12 * W.perturbation(xt.shape, 1.0, seed=19)
    z = np.zeros_like(xt)
    r = orc.switches_cross(q, gt, [(xt + e, z, b0), (xt - e, z, b0)], [np.zeros((3, 3))] * 2)
    assert r == {"support": 0, "clip": 0, "first": -1}

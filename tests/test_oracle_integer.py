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

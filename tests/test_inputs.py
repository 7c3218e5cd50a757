"""The seeded synthetic inputs (cq_inputs): grid order, supports of the initial fields,
the growing-mode screen and the batch recipe, as the input recipe states them."""
import math

import numpy as np
import pytest

import cq_inputs as ci


def test_grid_order():
    M = 5
    X, Y = ci.grid(M, 2)
    x = ci.grid_1d(M)
    assert np.allclose(x, np.arange(1, M + 1) / (M + 1))
    for iy in range(M):
        for ix in range(M):
            assert (X[iy * M + ix], Y[iy * M + ix]) == (x[ix], x[iy])          # dof = iy*M + ix
    X3, Y3, Z3 = ci.grid(3, 3)
    assert (X3[(2 * 3 + 1) * 3 + 0], Y3[(2 * 3 + 1) * 3 + 0], Z3[(2 * 3 + 1) * 3 + 0]) == (0.25, 0.5, 0.75)


def test_indicator_is_the_closed_quarter_box():
    """1D, 63 points, h = 1/64: the closed interval [1/4, 3/4] holds x_16 .. x_48."""
    g = ci.g0_indicator(63, 1)
    assert g.shape == (2, 63) and np.array_equal(g[0], g[1])
    assert np.array_equal(np.flatnonzero(g[0]) + 1, np.arange(16, 49))
    g2 = ci.g0_indicator(7, 2)                       # h = 1/8: x_2 .. x_6 per axis
    assert int(g2[0].sum()) == 25


def test_checkerboard_field():
    M, seed = 63, ci.SEED_BASE + 1
    g = ci.g0_checkerboard_uniform(M, seed)
    X, Y = ci.grid(M, 2)
    even = (np.floor(8 * X) + np.floor(8 * Y)) % 2 == 0
    assert g.shape == (2, M * M)
    assert np.all(g[:, ~even] == 0.0)
    assert np.all((g[:, even] > 0.0) & (g[:, even] < 1.0))
    assert not np.array_equal(g[0], g[1])                                      # two streams
    assert np.array_equal(g, ci.g0_checkerboard_uniform(M, seed))              # seeded
    assert not np.array_equal(g, ci.g0_checkerboard_uniform(M, seed + 1))


def test_disc_field():
    M = 127
    g = ci.g0_disc_gaussian(M, ci.SEED_BASE + 2)
    X, Y = ci.grid(M, 2)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    assert np.all(g[:, r2 > 0.0625 + 1e-9] == 0.0)
    inside = np.count_nonzero(g[0])
    assert abs(inside - math.pi * 0.0625 * (M + 1) ** 2) < 4 * (M + 1)      # area of the disc in cells
    assert abs(float(np.mean(g[0][r2 <= 0.0625]))) < 0.05                       # N(0,1) noise


def test_growth_rate_is_a_root():
    """The screen's rate solves (z^a1 + a + lam)(z^a2 + a + lam) = a^2 (a pole of the mode's
    transfer function); the 2D 255^2 workload with m = 0.49 has a fast-growing lowest mode,
    m = 0.4 and m > 1/2 have none."""
    lam = ci.lowest_eigenvalue(255, 2)
    assert lam == pytest.approx(2 * 4 * 256 ** 2 * math.sin(math.pi / 512) ** 2)
    z = ci.growth_rate(0.4, 0.6, 0.49, lam)
    a = (1 - 0.49) / (2 * 0.49 - 1)
    assert z > 100.0
    assert (z ** 0.4 + a + lam) * (z ** 0.6 + a + lam) == pytest.approx(a * a, rel=1e-9)
    assert ci.growth_rate(0.4, 0.6, 0.4, lam) == 0.0
    assert ci.growth_rate(0.4, 0.6, 0.7, lam) == 0.0


def test_batch_recipe():
    probs, fields, redraws = ci.batch_workload(24)
    assert len(probs) == len(fields) == 24 and redraws >= 0
    for p, g in zip(probs, fields):
        assert 0.1 <= p.alpha1 <= 0.9 and 0.1 <= p.alpha2 <= 0.9
        assert 0.30 <= p.m <= 0.48 or 0.52 <= p.m <= 0.70
        assert (p.dim == 1 and 31 <= p.M <= 1023) or (p.dim == 2 and 31 <= p.M <= 255)
        assert 512 <= p.N <= 8192 and p.form == ci.FAST and p.T == 1.0
        lam = ci.lowest_eigenvalue(p.M, p.dim)
        assert ci.growth_rate(p.alpha1, p.alpha2, p.m, lam) * p.T <= 600.0
        assert g.shape == (2, p.M ** p.dim) and np.all((g >= 0.0) & (g < 1.0))
    again = ci.batch_workload(24)[0]
    assert [(p.alpha1, p.M, p.N) for p in probs] == [(p.alpha1, p.M, p.N) for p in again]


def test_sample_indices():
    s = ci.sample_indices(1000, 50, 7)
    assert len(s) == 50 and np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < 1000
    assert np.array_equal(s, ci.sample_indices(1000, 50, 7))
    assert len(ci.sample_indices(10, 50, 7)) == 10

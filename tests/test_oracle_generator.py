"""Pins for the oracle's seeded instance generator (Sec. 2 random cubic
lattices; Sec. 3 random bicliques with couplings from [-1, 1]).  The laws of
the draws are fixed: +-1 fair coin, N(0,1), U(-1,1); values are FP32
numbers; different seeds give different instances; the layout of bonds is
checked through the energy of a planted state."""
import numpy as np
import pytest
from scipy import stats


def test_pm1_balance(orc):
    J = orc.gen_ea(16, orc.DIST_PM1, 1).reshape(-1)
    assert set(np.unique(J).tolist()) == {-1.0, 1.0}
    frac = (J > 0).mean()
    assert abs(frac - 0.5) < 4 * 0.5 / np.sqrt(J.size)
    Jb = orc.gen_biclique(128, orc.DIST_PM1, 3).reshape(-1)
    assert abs((Jb > 0).mean() - 0.5) < 4 * 0.5 / np.sqrt(Jb.size)


def test_gauss_law(orc):
    J = orc.gen_ea(16, orc.DIST_GAUSS, 2).reshape(-1)
    assert np.all(J.astype(np.float32).astype(np.float64) == J)
    _, p = stats.kstest(J, "norm")
    assert p > 1e-3
    assert abs(J.mean()) < 4 / np.sqrt(J.size)
    assert abs(J.var() - 1) < 4 * np.sqrt(2 / J.size)


def test_uniform_law(orc):
    J = orc.gen_biclique(128, orc.DIST_UNIF, 4).reshape(-1)
    assert J.min() > -1 and J.max() < 1
    assert np.all(J.astype(np.float32).astype(np.float64) == J)
    _, p = stats.kstest(J, "uniform", args=(-1, 2))
    assert p > 1e-3


def test_seeds_and_determinism(orc):
    a = orc.gen_ea(8, orc.DIST_PM1, 1)
    assert np.array_equal(a, orc.gen_ea(8, orc.DIST_PM1, 1))
    b = orc.gen_ea(8, orc.DIST_PM1, 2)
    assert (a != b).mean() > 0.4
    # neighbouring bonds are uncorrelated
    x = orc.gen_ea(16, orc.DIST_GAUSS, 9).reshape(-1)
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 4 / np.sqrt(x.size)


def test_biclique_prefix_consistency(orc):
    # bond e = i*n + j depends only on (seed, e): a smaller n reuses the leading stream
    big = orc.gen_biclique(8, orc.DIST_GAUSS, 5).reshape(-1)
    small = orc.gen_biclique(4, orc.DIST_GAUSS, 5).reshape(-1)
    assert np.array_equal(big[:16], small)

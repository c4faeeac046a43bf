"""The stationary law of the p-bit network (Sec. 1.2.1): for symmetric J the
update of Eqs. 2-3, in any update-group order, samples p(m) = e^{-beta E(m)}/Z.
Replicas run at fixed beta; their final states are independent samples and
are compared with the exact law from exhaustive enumeration (chi-square).  A
wrong sign, a dropped term, a wrong threshold rule or an update inside a colour
class would move the law far outside these tests."""
import numpy as np
import pytest
from scipy import stats


def _chi2_p(counts, probs, min_expected=5.0):
    n = counts.sum()
    exp = probs * n
    order = np.argsort(exp)
    c_s, e_s = counts[order], exp[order]
    # merge the smallest-expectation bins until each merged bin expects >= min_expected
    cc, ee, acc_c, acc_e = [], [], 0.0, 0.0
    for c, e in zip(c_s, e_s):
        acc_c += c; acc_e += e
        if acc_e >= min_expected:
            cc.append(acc_c); ee.append(acc_e); acc_c = acc_e = 0.0
    if acc_e > 0:
        cc[-1] += acc_c; ee[-1] += acc_e
    cc, ee = np.array(cc), np.array(ee)
    chi2 = ((cc - ee) ** 2 / ee).sum()
    return stats.chi2.sf(chi2, len(cc) - 1)


def _state_index(states):
    bits = (states > 0).astype(np.int64)
    return (bits << np.arange(states.shape[1], dtype=np.int64)).sum(axis=1)


@pytest.mark.parametrize("case,burn", [("ea_L2_gauss_h", 300), ("biclique_n4_gauss_h", 40)])
def test_full_state_law(orc, case, burn):
    # L=2 keeps its double bonds: strong couplings, two basins -> a longer burn-in to mix
    rng = np.random.default_rng(101)
    beta, R = 0.6, 40000
    if case.startswith("ea"):
        eu, ev, col = orc.ea_graph(2); N = 8
    else:
        eu, ev, col = orc.biclique_graph(4); N = 8
    J = rng.normal(size=eu.size)
    h = 0.5 * rng.normal(size=N)
    E = orc.brute_force(N, eu, ev, J, h)
    p = np.exp(-beta * (E - E.min())); p /= p.sum()
    out = orc.anneal(eu, ev, J, h, col, np.full(burn, beta), R, seed=77)
    idx = _state_index(out["final_state"])
    counts = np.bincount(idx, minlength=1 << N).astype(float)
    assert _chi2_p(counts, p) > 1e-4
    # and the reported energies are the energies of the states
    assert np.allclose(out["final_E"], E[idx])


def test_energy_level_law_n20(orc):
    # K_{10,10}, +-J: 2^20 states, compare the law of the energy levels
    n, beta, R, burn = 10, 0.25, 20000, 40
    eu, ev, col = orc.biclique_graph(n)
    J = orc.gen_biclique(n, orc.DIST_PM1, 21).reshape(-1)
    E = orc.brute_force(2 * n, eu, ev, J)
    levels, inv = np.unique(E, return_inverse=True)
    w = np.exp(-beta * (E - E.min()))
    p = np.bincount(inv, weights=w); p /= p.sum()
    out = orc.anneal(eu, ev, J, None, col, np.full(burn, beta), R, seed=5)
    k = np.searchsorted(levels, out["final_E"])
    assert np.all(levels[k] == out["final_E"])
    counts = np.bincount(k, minlength=levels.size).astype(float)
    assert _chi2_p(counts, p) > 1e-4


@pytest.mark.parametrize("beta,h", [(1.0, 0.3), (0.5, -1.2), (2.0, 0.05)])
def test_single_pbit_eq2(orc, beta, h):
    # an isolated p-bit in field h: P(m = +1) = 1/2 + tanh(beta h)/2 (Eq. 2)
    R = 200000
    out = orc.anneal(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.array([h]),
                     np.zeros(1, np.int32), np.array([beta]), R, seed=9)
    phat = (out["final_state"][:, 0] > 0).mean()
    p = 0.5 + 0.5 * np.tanh(beta * h)
    assert abs(phat - p) < 4.5 * np.sqrt(p * (1 - p) / R)

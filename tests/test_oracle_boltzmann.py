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


@pytest.mark.parametrize("graph", ["odd_cycle_chords_3col", "king_3x3_4col"])
def test_full_state_law_k_colours(orc, graph):
    """More than two update groups (Sec. 1.2.2 with a k-colouring): classes updated
    in colour order still sample the Boltzmann law."""
    rng = np.random.default_rng(202)
    beta, R, burn = 0.7, 40000, 60
    if graph.startswith("odd"):
        N = 9
        eu = list(range(9)) + [0, 2, 4]
        ev = [(i + 1) % 9 for i in range(9)] + [3, 5, 7]
        col = np.array([0, 1, 0, 1, 0, 1, 0, 1, 2], np.int32)  # 9-cycle needs a third colour
    else:
        N = 9
        eu, ev = [], []
        for y in range(3):
            for x in range(3):
                for dx, dy in ((1, 0), (0, 1), (1, 1), (-1, 1)):
                    X, Y = x + dx, y + dy
                    if 0 <= X < 3 and 0 <= Y < 3:
                        eu.append(y * 3 + x)
                        ev.append(Y * 3 + X)
        col = np.array([(x % 2) + 2 * (y % 2) for y in range(3) for x in range(3)], np.int32)
    eu, ev = np.array(eu, np.int32), np.array(ev, np.int32)
    assert orc.count_monochrome(eu, ev, col) == 0 and col.max() + 1 > 2
    J = rng.normal(size=eu.size)
    h = 0.5 * rng.normal(size=N)
    E = orc.brute_force(N, eu, ev, J, h)
    p = np.exp(-beta * (E - E.min())); p /= p.sum()
    out = orc.anneal(eu, ev, J, h, col, np.full(burn, beta), R, seed=91)
    idx = _state_index(out["final_state"])
    counts = np.bincount(idx, minlength=1 << N).astype(float)
    assert _chi2_p(counts, p) > 1e-4
    assert np.allclose(out["final_E"], E[idx])


def test_invalid_colouring_rejected(orc):
    eu, ev = np.array([0, 1], np.int32), np.array([1, 2], np.int32)
    with pytest.raises(ValueError):
        orc.anneal(eu, ev, np.ones(2), None, np.array([0, 0, 1], np.int32), np.full(3, 0.5), 2, seed=1)

"""Parallel tempering in the oracle (replica exchange, Hukushima & Nemoto 1996;
Sec. 6.1 names it): with one temperature it is fixed-beta annealing (checked
against the oracle's separate annealing loop), and with exchanges on, the slots
at the coldest temperature sample the Boltzmann law of that temperature (exact
enumeration, chi-square) -- an exchange rule with a wrong sign or a wrong
energy difference would bias that law."""
import numpy as np
import pytest
from scipy import stats


def _small(orc):
    eu, ev, col = orc.ea_graph(2)
    rng = np.random.default_rng(5)
    return eu, ev, col, rng.normal(size=eu.size), 0.4 * rng.normal(size=8)


def test_one_temperature_is_fixed_beta_annealing(orc):
    eu, ev, col, J, h = _small(orc)
    beta, S, R = 0.8, 30, 12
    pt = orc.anneal_pt(eu, ev, J, h, col, [beta], S, R, seed=3)
    ca = orc.anneal(eu, ev, J, h, col, np.full(S, beta), R, seed=3)
    for k in ("final_E", "best_E", "best_sweep", "final_state", "best_state"):
        assert np.array_equal(pt[k], ca[k]), k
    assert np.array_equal(pt["slot_temp"], np.zeros(R, np.int32))


def test_coldest_slots_sample_boltzmann(orc):
    eu, ev, col, J, h = _small(orc)
    ladder = np.array([0.2, 0.45, 0.7, 1.0])
    S, R, N = 300, 6000, 8
    pt = orc.anneal_pt(eu, ev, J, h, col, ladder, S, R, seed=17)
    cold = pt["slot_temp"] == ladder.size - 1
    assert cold.sum() == R  # one slot per chain at each temperature
    states = pt["final_state"][cold]
    idx = ((states > 0).astype(np.int64) << np.arange(N)).sum(axis=1)
    E = orc.brute_force(N, eu, ev, J, h)
    p = np.exp(-ladder[-1] * (E - E.min())); p /= p.sum()
    counts = np.bincount(idx, minlength=1 << N).astype(float)
    exp_ = p * R
    keep = exp_ >= 5
    chi2 = ((counts[keep] - exp_[keep]) ** 2 / exp_[keep]).sum() + \
        (counts[~keep].sum() - exp_[~keep].sum()) ** 2 / max(exp_[~keep].sum(), 1e-9)
    assert stats.chi2.sf(chi2, keep.sum()) > 1e-4
    assert np.all(pt["n_accept"] > 0)
    # the exchanges move temperatures: every temperature is held by exactly one slot per chain
    T = pt["slot_temp"].reshape(ladder.size, R)
    assert np.array_equal(np.sort(T, axis=0), np.repeat(np.arange(ladder.size)[:, None], R, axis=1))


def test_ladder_must_increase(orc):
    eu, ev, col, J, h = _small(orc)
    with pytest.raises(ValueError):
        orc.anneal_pt(eu, ev, J, h, col, [1.0, 0.5], 3, 2, seed=1)

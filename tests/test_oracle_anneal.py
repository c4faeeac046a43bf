"""Anneal-level pins for the oracle (Sec. 1.3.1 classical annealing with update
groups): incremental energy (Eq. 3) equals recomputed energy every sweep;
annealing reaches exhaustive-search and closed-form ground states; the best
state is the running minimum; replicas are independent of how many run."""
import numpy as np
import pytest


def _sched(orc, S, b0=0.1, b1=4.0):
    return orc.schedule(orc.SCHED_LINEAR, b0, b1, S)


@pytest.mark.parametrize("dist", [0, 1])
def test_incremental_equals_recomputed(orc, dist):
    L = 4
    J = orc.gen_ea(L, dist, 3)
    h = None if dist == 0 else np.random.default_rng(1).normal(size=L ** 3)
    out = orc.anneal_ea(L, J, h, _sched(orc, 60), R=6, seed=1)
    if dist == 0:
        assert out["max_incr_err"] == 0.0
    else:
        assert out["max_incr_err"] < 1e-9


def test_reaches_brute_force_ground_state(orc):
    n = 8
    eu, ev, col = orc.biclique_graph(n)
    J = orc.gen_biclique(n, orc.DIST_GAUSS, 31).reshape(-1)
    E0 = orc.brute_force(2 * n, eu, ev, J).min()
    out = orc.anneal(eu, ev, J, None, col, _sched(orc, 400, 0.1, 5.0), R=32, seed=2)
    assert out["best_E"].min() == pytest.approx(E0, abs=1e-9)
    assert np.all(out["best_E"] >= E0 - 1e-9)


def test_ferro_biclique_closed_form(orc):
    n = 32
    J = np.ones((n, n))
    out = orc.anneal_biclique(n, J, None, _sched(orc, 200, 0.05, 3.0), R=8, seed=3)
    assert np.all(out["best_E"] == -n * n)
    for s in out["best_state"]:
        assert abs(int(s.astype(int).sum())) == 2 * n


def test_mattis_ground_state(orc):
    rng = np.random.default_rng(8)
    L = 4; N = 64
    eu, ev, col = orc.ea_graph(L)
    xi = rng.choice([-1, 1], size=N).astype(np.int8)
    J = xi[eu].astype(float) * xi[ev]
    out = orc.anneal_ea(L, J, None, _sched(orc, 300, 0.1, 3.0), R=8, seed=4)
    assert np.all(out["best_E"] == -3 * N)
    for s in out["best_state"]:
        assert np.array_equal(s, xi) or np.array_equal(s, -xi)


def test_best_is_running_minimum(orc):
    L = 4
    J = orc.gen_ea(L, orc.DIST_PM1, 5)
    out = orc.anneal_ea(L, J, None, _sched(orc, 80), R=5, seed=6, trace=True)
    eu, ev, _ = orc.ea_graph(L)
    tr = out["trace_E"]
    for r in range(5):
        s = out["best_sweep"][r]
        assert out["best_E"][r] == min(tr[r].min(), orc.energy(eu, ev, J, None, out["best_state"][r]))
        assert s >= 0 and tr[r, s] == out["best_E"][r]
        assert np.all(tr[r, :s] > out["best_E"][r])      # strictly: the earliest sweep is kept
        assert orc.energy(eu, ev, J, None, out["best_state"][r]) == out["best_E"][r]
        assert orc.energy(eu, ev, J, None, out["final_state"][r]) == out["final_E"][r] == tr[r, -1]


def test_replicas_independent_of_count(orc):
    L = 4
    J = orc.gen_ea(L, orc.DIST_PM1, 7)
    a = orc.anneal_ea(L, J, None, _sched(orc, 30), R=9, seed=11)
    b = orc.anneal_ea(L, J, None, _sched(orc, 30), R=3, seed=11)
    assert np.array_equal(a["final_state"][:3], b["final_state"])
    assert np.array_equal(a["best_sweep"][:3], b["best_sweep"])


def test_zero_sweeps(orc):
    L = 2
    J = orc.gen_ea(L, orc.DIST_PM1, 1)
    out = orc.anneal_ea(L, J, None, np.zeros(0), R=4, seed=1)
    assert np.array_equal(out["final_state"], out["best_state"])
    assert np.all(out["best_sweep"] == -1)
    assert np.array_equal(out["final_E"], out["best_E"])


def test_initial_state_fair(orc):
    L = 8
    J = orc.gen_ea(L, orc.DIST_PM1, 1)
    out = orc.anneal_ea(L, J, None, np.zeros(0), R=64, seed=3)
    frac = (out["final_state"] > 0).mean()
    assert abs(frac - 0.5) < 4 * 0.5 / np.sqrt(out["final_state"].size)


def test_bad_colouring_rejected(orc):
    with pytest.raises(ValueError):
        orc.anneal_ea(3, orc.gen_ea(3, 0, 1), None, np.zeros(1), R=1, seed=1)
    eu, ev, col = orc.biclique_graph(3)
    col[0] = 1
    with pytest.raises(ValueError):
        orc.anneal(eu, ev, np.ones(9), None, col, np.zeros(1), 1, 1)

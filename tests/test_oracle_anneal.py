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


def _iterate_class_steps(orc, eu, ev, J, h, col, betas, R, seed, r_first=0):
    """Initial state of the anneal (zero sweeps), then every class of every sweep by class_step."""
    k = int(col.max()) + 1
    m = orc.anneal(eu, ev, J, h, col, np.zeros(0), R, seed, n_colours=k, r_first=r_first)["final_state"]
    for s, beta in enumerate(betas):
        for c in range(k):
            m = orc.class_step(eu, ev, J, h, col, c, beta, s, m, seed, r_first=r_first, n_colours=k)["state"]
    return m


@pytest.mark.parametrize("kind", ["ea_pm1_h", "ea_gauss_h", "biclique_unif", "three_colour"])
def test_class_steps_replay_the_anneal(orc, kind):
    """The one-class step reproduces the annealing loop: iterating it over every class of
    every sweep from the initial state gives the anneal's final state, replica for replica
    (replicas offset by r_first so the counters' replica words are exercised)."""
    rng = np.random.default_rng(5)
    if kind.startswith("ea"):
        L = 4
        eu, ev, col = orc.ea_graph(L)
        J = orc.gen_ea(L, orc.DIST_PM1 if "pm1" in kind else orc.DIST_GAUSS, 9).reshape(-1)
        h = rng.integers(-2, 3, size=L ** 3).astype(float) if "pm1" in kind else rng.normal(size=L ** 3)
    elif kind == "biclique_unif":
        n = 6
        eu, ev, col = orc.biclique_graph(n)
        J = orc.gen_biclique(n, orc.DIST_UNIF, 4).reshape(-1)
        h = None
    else:  # 5-cycle with a chord: 3 colours
        eu = np.array([0, 1, 2, 3, 4, 0], np.int32)
        ev = np.array([1, 2, 3, 4, 0, 2], np.int32)
        col = np.array([0, 1, 2, 0, 1], np.int32)
        J = rng.normal(size=6)
        h = rng.normal(size=5)
    betas = orc.schedule(orc.SCHED_GEOMETRIC, 0.1, 4.0, 25)
    R, seed, r0 = 6, 17, 5
    ref = orc.anneal(eu, ev, J, h, col, betas, R, seed, n_colours=int(col.max()) + 1, r_first=r0)
    got = _iterate_class_steps(orc, eu, ev, J, h, col, betas, R, seed, r_first=r0)
    assert np.array_equal(got, ref["final_state"])


def test_class_step_outputs(orc):
    """Only the stepped class changes; P is the p-bit law of the spin's field and the
    new spin is +1 exactly when the word is below floor(P 2^32)."""
    L = 4
    eu, ev, col = orc.ea_graph(L)
    J = orc.gen_ea(L, orc.DIST_GAUSS, 2).reshape(-1)
    m0 = np.random.default_rng(3).choice(np.array([-1, 1], np.int8), size=(3, L ** 3))
    out = orc.class_step(eu, ev, J, None, col, 1, 0.7, 4, m0, 8)
    assert np.array_equal(out["state"][:, col == 0], m0[:, col == 0])
    assert np.all(np.isnan(out["P"][:, col == 0])) and np.all(out["w"][:, col == 0] == 0)
    for r in range(3):
        F = orc.fields(eu, ev, J, None, m0[r])
        for i in np.flatnonzero(col == 1)[:20]:
            P = 0.5 + 0.5 * np.tanh(0.7 * F[i])
            assert out["P"][r, i] == pytest.approx(P, rel=0, abs=1e-15)  # libm vs numpy tanh: last ulps
            T = min(int(np.floor(out["P"][r, i] * 2.0 ** 32)), 2 ** 32 - 1)
            assert out["state"][r, i] == (1 if int(out["w"][r, i]) < T else -1)

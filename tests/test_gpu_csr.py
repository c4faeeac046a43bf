"""GPU parity of the general sparse (CSR, k-colour) path against the CPU oracle.

+-1 couplings: bit-exact trajectories (final/best states and energies, best
sweep) for 3-, 4- and 5-colour graphs, with the library's greedy colouring and
with a given colouring.  Real couplings: fields within 1e-5 of FP64 relative to
sum_j |J_ij| + |h_i|, returned-state energies within 1e-9 relative, ensemble
mean energy per spin within 3 standard errors.
"""
import math

import numpy as np
import pytest

import synth_inputs as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def _graph(name):
    if name == "cube5":
        return 125, syn.graph_periodic_cube(5)
    if name == "king12x10":
        return 120, syn.graph_king(12, 10)
    if name == "random300":
        return 300, syn.graph_random(300, 1200, 3)
    if name == "dense80":
        return 80, syn.graph_random(80, 1500, 4)
    raise KeyError(name)


def _run(pb, N, eu, ev, J, h, colour, sc, R, seed):
    inst = pb.pb_create_graph_instance(N, eu, ev, J, h, colour)
    try:
        k = pb.pb_instance_colours(inst)
        run = pb.pb_anneal(inst, sc, R, seed)
        try:
            fe, be, bs = pb.pb_energy(run, R)
            out = dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb.pb_final_states(run, R, N),
                       best_state=pb.pb_best_states(run, R, N))
        finally:
            pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)
    return out, k


CASES = [
    # graph, R, S, kind, b0, b1, hmax, seed, greedy
    ("cube5", 8, 40, 0, 0.1, 3.0, 0, 1, True),
    ("king12x10", 37, 25, 1, 0.1, 5.0, 2, 2, True),
    ("random300", 64, 15, 0, 0.35, 3.5, 0, 3, True),
    ("dense80", 5, 30, 0, 0.05, 2.0, 1, 4, True),
    ("cube5", 3, 12, 0, 0.5, 0.5, 0, 5, False),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}R{c[1]}S{c[2]}h{c[6]}{'g' if c[8] else 'c'}" for c in CASES])
def test_pm1_bit_exact(pb, orc, case):
    name, R, S, kind, b0, b1, hmax, seed, greedy = case
    N, (eu, ev) = _graph(name)
    J = syn.edge_couplings(eu.size, "pm1", seed)
    h = syn.int_fields(N, hmax, seed + 1) if hmax else None
    if greedy:
        col, k = pb.pb_greedy_colouring(N, eu, ev)
    else:
        # a different proper colouring: the greedy classes in reverse order
        col, k = pb.pb_greedy_colouring(N, eu, ev)
        col = (k - 1 - col).astype(np.int32)  # reversed class order
    g, kg = _run(pb, N, eu, ev, J, h, None if greedy else col, pb.make_schedule(kind, S, b0, b1), R, seed)
    assert kg == k and k >= 3
    o = orc.anneal(eu, ev, J.astype(np.float64), None if h is None else h.astype(np.float64), col,
                   orc.schedule(kind, b0, b1, S), R, seed, n_colours=k)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[key], o[key]), key


@pytest.mark.parametrize("variant", ["isolated", "degree9"])
def test_pm1_padded_row_limits(pb, orc, variant):
    """The padded-row form (+-1, degree <= 8) at its edges: spins with no
    neighbour (every slot names the zero row; F = h) and, one past the limit, a
    hub of degree 9 (the compressed-row form); bit-exact against the oracle."""
    N0 = 120
    eu, ev = syn.graph_king(12, 10)
    if variant == "isolated":
        N = N0 + 7  # seven spins without edges
    else:
        N = N0 + 1  # a hub joined to 9 spins of the king graph
        hub = np.full(9, N0, np.int32)
        eu = np.concatenate([eu, hub])
        ev = np.concatenate([ev, np.arange(0, 90, 10, dtype=np.int32)])
    J = syn.edge_couplings(eu.size, "pm1", 91)
    h = syn.int_fields(N, 3, 92)
    col, k = pb.pb_greedy_colouring(N, eu, ev)
    R, S = 21, 18
    g, kg = _run(pb, N, eu, ev, J, h, None, pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.1, 3.0), R, 93)
    assert kg == k
    o = orc.anneal(eu, ev, J.astype(np.float64), h.astype(np.float64), col, orc.schedule(orc.SCHED_LINEAR, 0.1, 3.0, S),
                   R, 93, n_colours=k)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[key], o[key]), key


def test_bench_size_sampled(pb, orc):
    """The general-graph bench configuration: odd periodic cube L = 25 (4 greedy
    colours), +-1, 1024 replicas (256 replica words), 20 sweeps; replicas 0, 513
    and 1023 replayed one by one on the oracle, bit-exact."""
    L, R, S = 25, 1024, 20
    N = L ** 3
    eu, ev = syn.graph_periodic_cube(L)
    J = syn.edge_couplings(eu.size, "pm1", 61)
    col, k = pb.pb_greedy_colouring(N, eu, ev)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    g, kg = _run(pb, N, eu, ev, J, None, None, sc, R, 67)
    assert kg == k
    ob = orc.schedule(orc.SCHED_LINEAR, 0.1, 3.0, S)
    for r in (0, 513, 1023):
        o = orc.anneal(eu, ev, J.astype(np.float64), None, col, ob, 1, 67, n_colours=k, r_first=r)
        for key in ("final_state", "best_state"):
            assert np.array_equal(o[key][0], g[key][r]), (r, key)
        assert o["best_E"][0] == g["best_E"][r] and o["best_sweep"][0] == g["best_sweep"][r]
        assert o["final_E"][0] == g["final_E"][r]


def _read_run(pb, run, R, N):
    fe, be, bs = pb.pb_energy(run, R)
    return dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb.pb_final_states(run, R, N),
                best_state=pb.pb_best_states(run, R, N))


@pytest.mark.parametrize("name,s0", [("cube5", 17), ("king12x10", 1), ("biclique24", 29), ("cube5", 0),
                                     ("random300", 40)])
def test_resume_split_equals_one_run(pb, orc, name, s0):
    """Checkpoint / resume: sweeps 0..s0-1, then pb_anneal_resume from that run's final
    state and running best, equal one uninterrupted run bit for bit (+-1 couplings)."""
    if name == "biclique24":
        n = 24
        eu, ev, _ = orc.biclique_graph(n)
        N = 2 * n
    else:
        N, (eu, ev) = _graph(name)
    R, S, seed = 37, 40, 3
    J = syn.edge_couplings(eu.size, "pm1", 90 + s0)
    h = syn.int_fields(N, 2, 5) if name == "king12x10" else None
    betas = orc.schedule(orc.SCHED_LINEAR, 0.1, 3.0, S)
    full = pb.make_schedule(pb.PB_SCHED_EXPLICIT, S, betas=betas)
    first = pb.make_schedule(pb.PB_SCHED_EXPLICIT, s0, betas=betas[:s0] if s0 else None)
    inst = pb.pb_create_graph_instance(N, eu, ev, J, h)
    try:
        runs = []
        try:
            runs.append(pb.pb_anneal(inst, full, R, seed))
            one = _read_run(pb, runs[-1], R, N)
            runs.append(pb.pb_anneal(inst, first, R, seed))
            a = _read_run(pb, runs[-1], R, N)
            runs.append(pb.pb_anneal_resume(inst, full, R, seed, s0, a["final_state"], a["best_state"], a["best_E"],
                                            a["best_sweep"]))
            b = _read_run(pb, runs[-1], R, N)
        finally:
            for r in runs:
                pb.pb_run_destroy(r)
        for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
            assert np.array_equal(b[key], one[key]), key
    finally:
        pb.pb_instance_destroy(inst)


def test_resume_errors(pb):
    N, (eu, ev) = _graph("cube5")
    J = syn.edge_couplings(eu.size, "pm1", 1)
    inst = pb.pb_create_graph_instance(N, eu, ev, J)
    try:
        sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 10, 0.1, 1.0)
        st = np.ones((4, N), np.int8)
        be = np.zeros(4)
        bs = np.full(4, -1, np.int32)
        with pytest.raises(pb.PbError, match="PB_EINVAL"):
            pb.pb_anneal_resume(inst, sc, 4, 1, 11, st, st, be, bs)       # first_sweep beyond the schedule
        with pytest.raises(pb.PbError, match="PB_EINVAL"):
            pb.pb_anneal_resume(inst, sc, 4, 1, 3, st, st, be, np.full(4, 3, np.int32))  # best after first_sweep
        bad = st.copy()
        bad[1, 7] = 0
        with pytest.raises(pb.PbError, match="PB_EINVAL"):
            pb.pb_anneal_resume(inst, sc, 4, 1, 3, bad, st, be, bs)       # not a +-1 state
    finally:
        pb.pb_instance_destroy(inst)
    Jb = pb.pb_generate_biclique(16, pb.PB_DIST_PM1, 2)
    binst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, Jb, None, n=16)
    try:
        with pytest.raises(pb.PbError, match="PB_EUNSUPPORTED"):
            pb.pb_anneal_resume(binst, sc, 4, 1, 3, np.ones((4, 32), np.int8), np.ones((4, 32), np.int8), be, bs)
    finally:
        pb.pb_instance_destroy(binst)


def test_f32_fields(pb, orc):
    N, (eu, ev) = _graph("random300")
    J = syn.edge_couplings(eu.size, "gauss", 11)
    h = syn.real_fields(N, 0.5, 12)
    inst = pb.pb_create_graph_instance(N, eu, ev, J, h)
    try:
        m = syn.states(6, N, 13)
        F = pb.pb_fields(inst, m)
    finally:
        pb.pb_instance_destroy(inst)
    Jd, hd = J.astype(np.float64), h.astype(np.float64)
    scale = orc.fields(eu, ev, np.abs(Jd), np.abs(hd), np.ones(N, np.int8))
    for r in range(6):
        assert np.all(np.abs(F[r] - orc.fields(eu, ev, Jd, hd, m[r])) <= 1e-5 * scale)


def test_f32_energies_and_ensemble(pb, orc):
    N, (eu, ev) = _graph("king12x10")
    J = syn.edge_couplings(eu.size, "unif", 21)
    R, S = 256, 60
    col, k = pb.pb_greedy_colouring(N, eu, ev)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g, _ = _run(pb, N, eu, ev, J, None, None, sc, R, 5)
    Jd = J.astype(np.float64)
    for r in range(R):
        e = orc.energy(eu, ev, Jd, None, g["best_state"][r])
        assert abs(g["best_E"][r] - e) <= 1e-9 * abs(e)
    o = orc.anneal(eu, ev, Jd, None, col, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), R, 5, n_colours=k)
    eg, eo = g["final_E"] / N, o["final_E"] / N
    se = math.sqrt(eg.var(ddof=1) / R + eo.var(ddof=1) / R)
    assert abs(eg.mean() - eo.mean()) <= 3 * se + 1e-12


def test_colouring_errors(pb):
    eu, ev = np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32)
    J = np.ones(3, np.int8)
    with pytest.raises(pb.PbError, match="PB_ECOLOUR"):
        pb.pb_create_graph_instance(3, eu, ev, J, None, np.array([0, 1, 1], np.int32))
    with pytest.raises(pb.PbError, match="PB_EINVAL"):
        pb.pb_create_graph_instance(3, np.array([0], np.int32), np.array([0], np.int32), np.ones(1, np.int8))
    with pytest.raises(pb.PbError, match="PB_EINVAL"):
        pb.pb_create_graph_instance(3, eu, ev, np.array([1, 2, 1], np.int8))


def test_csr_in_batch_equals_alone(pb):
    N, (eu, ev) = _graph("cube5")
    J = syn.edge_couplings(eu.size, "pm1", 31)
    inst = pb.pb_create_graph_instance(N, eu, ev, J)
    Jb = pb.pb_generate_biclique(64, pb.PB_DIST_PM1, 32)
    binst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, Jb, None, n=64)
    try:
        sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 20, 0.1, 3.0)
        runs = pb.pb_anneal_batch([inst, binst], [sc, sc], [32, 16], [7, 8])
        try:
            fe, be, bs = pb.pb_energy(runs[0], 32)
            st = pb.pb_best_states(runs[0], 32, N)
        finally:
            for r in runs:
                pb.pb_run_destroy(r)
        run = pb.pb_anneal(inst, sc, 32, 7)
        try:
            fe2, be2, bs2 = pb.pb_energy(run, 32)
            st2 = pb.pb_best_states(run, 32, N)
        finally:
            pb.pb_run_destroy(run)
        assert np.array_equal(fe, fe2) and np.array_equal(be, be2) and np.array_equal(bs, bs2)
        assert np.array_equal(st, st2)
    finally:
        pb.pb_instance_destroy(inst)
        pb.pb_instance_destroy(binst)


def test_sparsified_bench_size_sampled(pb, orc):
    """The sparsified-biclique bench configuration: +-1 K_{512,512} as a copy graph
    (at most 4 edges per copy, copy strength 2: 131072 spins), 256 replicas, 30
    sweeps; replicas 0 and 255 replayed one by one on the oracle, bit-exact."""
    n, R, S = 512, 256, 30
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 61)
    sp = pb.pb_sparsify_biclique(J, 4, 2)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g, k = _run(pb, sp["N"], sp["eu"], sp["ev"], sp["J"], None, sp["colour"], sc, R, 13)
    assert k == 2
    ob = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S)
    for r in (0, 255):
        o = orc.anneal(sp["eu"], sp["ev"], sp["J"].astype(np.float64), None, sp["colour"], ob, 1, 13, n_colours=2,
                       r_first=r)
        for key in ("final_state", "best_state"):
            assert np.array_equal(o[key][0], g[key][r]), (r, key)
        assert o["best_E"][0] == g["best_E"][r] and o["best_sweep"][0] == g["best_sweep"][r]


@pytest.mark.parametrize("n,cs", [(24, 2), (17, 3)])
def test_sparsified_biclique_bit_exact(pb, orc, n, cs):
    """The copy graph of a +-J biclique (degree <= 6, two update groups) on the CSR
    path, with the construction's own colouring, against the oracle."""
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 50 + n)
    sp = pb.pb_sparsify_biclique(J, 4, cs)
    R, S = 20, 30
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g, k = _run(pb, sp["N"], sp["eu"], sp["ev"], sp["J"], None, sp["colour"], sc, R, 11)
    assert k == 2
    o = orc.anneal(sp["eu"], sp["ev"], sp["J"].astype(np.float64), None, sp["colour"],
                   orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), R, 11, n_colours=2)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[key], o[key]), key
    # projected best states are biclique states; their energies from the oracle
    proj = pb.pb_sparse_project(sp["copy_of"], 2 * n, g["best_state"])
    beu, bev, _ = orc.biclique_graph(n)
    e = [orc.energy(beu, bev, J.astype(np.float64).reshape(-1), None, proj[r]) for r in range(R)]
    assert min(e) >= -n * n

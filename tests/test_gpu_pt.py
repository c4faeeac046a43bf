"""Parallel tempering on the GPU against the oracle: +-J runs are bit-exact per
slot (states, energies, best sweeps), with the same final temperature of every
slot and the same accepted exchanges per pair; real couplings agree in the mean
energy at every temperature within 3 standard errors."""
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


def _graph(pb, name):
    if name == "cube4":
        eu, ev = syn.graph_periodic_cube(4)
        return 64, eu, ev
    if name == "king10x8":
        eu, ev = syn.graph_king(10, 8)
        return 80, eu, ev
    if name == "random120":
        eu, ev = syn.graph_random(120, 300, 9)
        return 120, eu, ev
    raise KeyError(name)


def _pt(pb, N, eu, ev, J, h, ladder, S, C, seed):
    inst = pb.pb_create_graph_instance(N, eu, ev, J, h)
    try:
        col, k = pb.pb_greedy_colouring(N, eu, ev)
        run = pb.pb_anneal_pt(inst, ladder, S, C, seed)
        try:
            G = len(ladder) * C
            fe, be, bs = pb.pb_energy(run, G)
            temp, acc = pb.pb_pt_state(run, len(ladder), C)
            out = dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb.pb_final_states(run, G, N),
                       best_state=pb.pb_best_states(run, G, N), slot_temp=temp, n_accept=acc)
        finally:
            pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)
    return out, col, k


@pytest.mark.parametrize("graph,M,C,S,hmax", [("cube4", 4, 5, 30, 0), ("king10x8", 7, 16, 25, 1),
                                              ("random120", 1, 9, 20, 0), ("cube4", 2, 3, 40, 2)])
def test_pm1_bit_exact(pb, orc, graph, M, C, S, hmax):
    N, eu, ev = _graph(pb, graph)
    J = syn.edge_couplings(eu.size, "pm1", M + C)
    h = syn.int_fields(N, hmax, 3) if hmax else None
    ladder = np.array([0.9]) if M == 1 else (np.array([0.8, 1.0]) if M == 2 else np.linspace(0.2, 1.5, M))
    g, col, k = _pt(pb, N, eu, ev, J, h, ladder, S, C, 21)
    o = orc.anneal_pt(eu, ev, J.astype(np.float64), None if h is None else h.astype(np.float64), col, ladder, S, C,
                      21, n_colours=k)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep", "slot_temp", "n_accept"):
        assert np.array_equal(g[key], o[key]), key
    if M > 1:
        assert g["n_accept"].sum() > 0


def test_bench_configuration_bit_exact(pb, orc):
    """The tempering bench configuration: periodic cube L = 25 (4 greedy colours),
    +-1, linear ladder 0.1 .. 3.0 with 16 rungs x 64 chains (1024 slots); 10 sweeps,
    every slot bit-exact (states, energies, final temperatures, accepted exchanges)."""
    L, C, S = 25, 64, 10
    N = L ** 3
    eu, ev = syn.graph_periodic_cube(L)
    J = syn.edge_couplings(eu.size, "pm1", 77)
    ladder = np.linspace(0.1, 3.0, 16)
    g, col, k = _pt(pb, N, eu, ev, J, None, ladder, S, C, 9)
    o = orc.anneal_pt(eu, ev, J.astype(np.float64), None, col, ladder, S, C, 9, n_colours=k)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep", "slot_temp", "n_accept"):
        assert np.array_equal(g[key], o[key]), key
    assert g["n_accept"].sum() > 0


def test_f32_mean_energy_per_temperature(pb, orc):
    N, eu, ev = _graph(pb, "king10x8")
    J = syn.edge_couplings(eu.size, "gauss", 5)
    ladder = np.array([0.3, 0.6, 1.0, 1.6])
    C, S = 96, 60
    g, col, k = _pt(pb, N, eu, ev, J, None, ladder, S, C, 8)
    o = orc.anneal_pt(eu, ev, J.astype(np.float64), None, col, ladder, S, C, 8, n_colours=k)
    for t in range(ladder.size):
        eg = g["final_E"][g["slot_temp"] == t] / N
        eo = o["final_E"][o["slot_temp"] == t] / N
        assert eg.size == C and eo.size == C
        se = math.sqrt(eg.var(ddof=1) / C + eo.var(ddof=1) / C)
        assert abs(eg.mean() - eo.mean()) <= 3 * se + 1e-12, t
    # returned energies are those of the returned states (FP64)
    for q in range(0, ladder.size * C, 37):
        e = orc.energy(eu, ev, J.astype(np.float64), None, g["best_state"][q])
        assert abs(g["best_E"][q] - e) <= 1e-9 * abs(e)


def test_pt_errors(pb):
    N, eu, ev = _graph(pb, "cube4")
    inst = pb.pb_create_graph_instance(N, eu, ev, syn.edge_couplings(eu.size, "pm1", 1))
    try:
        with pytest.raises(pb.PbError, match="PB_EINVAL"):
            pb.pb_anneal_pt(inst, [1.0, 0.5], 3, 2, 1)
    finally:
        pb.pb_instance_destroy(inst)
    J = pb.pb_generate_ea(4, pb.PB_DIST_PM1, 1)
    ea = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=4)
    try:
        with pytest.raises(pb.PbError, match="PB_EUNSUPPORTED"):
            pb.pb_anneal_pt(ea, [0.5, 1.0], 3, 2, 1)
    finally:
        pb.pb_instance_destroy(ea)

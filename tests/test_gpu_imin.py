"""The batched Algorithm 1 driver (Sec. 4.1.3) returns the same minimal budget
as the oracle's sequential loop with early exit, for +-J instances (whose
trials are bit-exact on both sides), whatever the number of budgets per launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


@pytest.mark.parametrize("topo", ["ea4", "biclique16", "csr_cube3"])
@pytest.mark.parametrize("per", [1, 3, 8])
def test_imin_matches_oracle(pb, orc, topo, per):
    rng = np.random.default_rng(7)
    if topo == "ea4":
        L = 4
        J = pb.pb_generate_ea(L, pb.PB_DIST_PM1, 41)
        inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L)
        eu, ev, col = orc.ea_graph(L)
        Jd = J.astype(np.float64).reshape(-1)
    elif topo == "biclique16":
        n = 16
        J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 42)
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n)
        eu, ev, col = orc.biclique_graph(n)
        Jd = J.astype(np.float64).reshape(-1)
    else:
        import synth_inputs as syn
        eu, ev = syn.graph_periodic_cube(3)
        J = syn.edge_couplings(eu.size, "pm1", 43)
        inst = pb.pb_create_graph_instance(27, eu, ev, J)
        col, _ = pb.pb_greedy_colouring(27, eu, ev)
        Jd = J.astype(np.float64)
    try:
        k = pb.pb_instance_colours(inst)
        G = orc.anneal(eu, ev, Jd, None, col, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, 300), 32, 3,
                       n_colours=k)["best_E"].min()
        for p, ps in ((0.97, 0.8), (1.0, 0.5)):
            r = pb.pb_find_imin(inst, G, p, ps, i_start=2, i_step=3, trials=16, i_max=60, budgets_per_launch=per,
                                seed=1000)
            o = orc.find_imin(eu, ev, Jd, None, col, G, p, ps, 2, 3, trials=16, beta_i=0.35, beta_f=3.5, i_max=60,
                              seed=1000, n_colours=k)
            assert (r.i_min if r.i_min >= 0 else None) == o, (p, ps)
            if r.i_min >= 0:
                assert r.budgets_tried == (r.i_min - 2) // 3 + 1
    finally:
        pb.pb_instance_destroy(inst)

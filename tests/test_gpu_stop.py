"""Stop at the target (PB_FLAG_STOP_AT_TARGET; the quality criterion of Sec. 1.3.1,
Fig. 1): every replica's running best freezes at its first sweep whose energy is at
or below the target, and a run ends early once every replica has reached it.

+-1 couplings, against the oracle: the oracle's full run gives each replica's first
sweep at the target (its trace); the expected best energy, sweep and state of a
replica that reached it are those of the oracle's run cut right after that sweep,
otherwise those of the full run.  Bit-exact in every form, alone and in a batch."""
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


def _expected(orc, eu, ev, J, h, col, betas, R, seed, target):
    k = int(col.max()) + 1
    full = orc.anneal(eu, ev, J, h, col, betas, R, seed, n_colours=k, trace=True)
    hit = np.array([int(np.argmax(tr <= target)) if (tr <= target).any() else -1 for tr in full["trace_E"]])
    exp = {key: full[key].copy() for key in ("best_E", "best_sweep", "best_state")}
    for r in np.flatnonzero(hit >= 0):
        cut = orc.anneal(eu, ev, J, h, col, betas[: hit[r] + 1], 1, seed, n_colours=k, r_first=int(r))
        for key in exp:
            exp[key][r] = cut[key][0]
    return exp, hit, full


def _gpu_run(pb, inst, sched, R, seed, form, target):
    run = pb.pb_anneal(inst, sched, R, seed, pb.make_opts(form, target, pb.PB_FLAG_STOP_AT_TARGET))
    try:
        N = pb.pb_instance_spins(inst)
        fe, be, bs = pb.pb_energy(run, R)
        return dict(best_E=be, best_sweep=bs, best_state=pb.pb_best_states(run, R, N),
                    target_sweep=pb.pb_target_sweeps(run, R), final_E=fe, device_ms=pb.pb_run_device_ms(run))
    finally:
        pb.pb_run_destroy(run)


def _check(g, exp, hit):
    assert np.array_equal(g["target_sweep"], hit)
    for key in ("best_E", "best_sweep", "best_state"):
        assert np.array_equal(g[key], exp[key]), key
    assert 0 < (hit >= 0).sum() < hit.size  # the case exercises both kinds of replica


CASES = [
    # topology, size, R, S, form
    ("ea", 8, 24, 60, "plain"),
    ("ea", 8, 24, 60, "resident"),       # generic tile
    ("ea", 32, 8, 40, "resident"),       # fast tile L = 32
    ("ea", 16, 40, 50, "resident"),      # generic tile with WT > 1 after splitting, fields
    ("bq", 64, 40, 60, "tensor"),
    ("bq", 64, 40, 60, "cudacore"),
    ("bq", 64, 40, 60, "resident"),
    ("csr", 5, 36, 50, "plain"),         # odd periodic cube: greedy colours
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}{c[1]}R{c[2]}{c[4]}" for c in CASES])
def test_stop_at_target_bit_exact(pb, orc, case):
    topo, size, R, S, form = case
    seed = 41
    betas = orc.schedule(orc.SCHED_GEOMETRIC, 0.1, 5.0, S)
    sched = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
    h = None
    if topo == "ea":
        J = syn.ea_couplings(size, "pm1", 3 + size)
        if size == 16:
            h = syn.int_fields(size ** 3, 2, 5)
        inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=size)
        eu, ev, col = orc.ea_graph(size)
        Jd = J.astype(np.float64).reshape(-1)
    elif topo == "bq":
        J = syn.biclique_couplings(size, "pm1", 7)
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=size)
        eu, ev, col = orc.biclique_graph(size)
        Jd = J.astype(np.float64).reshape(-1)
    else:
        eu, ev = syn.graph_periodic_cube(size)
        Jc = syn.edge_couplings(eu.size, "pm1", 9)
        col, _ = pb.pb_greedy_colouring(size ** 3, eu, ev)
        inst = pb.pb_create_graph_instance(size ** 3, eu, ev, Jc, None, col)
        Jd = Jc.astype(np.float64)
    form_id = {"plain": pb.PB_FORM_PLAIN, "resident": pb.PB_FORM_RESIDENT, "tensor": pb.PB_FORM_TENSOR,
               "cudacore": pb.PB_FORM_CUDACORE}[form]
    try:
        hd = None if h is None else h.astype(np.float64)
        full = orc.anneal(eu, ev, Jd, hd, np.asarray(col, np.int32), betas, R, seed,
                          n_colours=int(np.max(col)) + 1)
        target = float(np.median(full["best_E"]))    # about half the replicas reach it
        exp, hit, _ = _expected(orc, eu, ev, Jd, hd, np.asarray(col, np.int32), betas, R, seed, target)
        g = _gpu_run(pb, inst, sched, R, seed, form_id, target)
    finally:
        pb.pb_instance_destroy(inst)
    _check(g, exp, hit)


def test_stop_at_target_in_a_batch(pb, orc):
    """The same stop-mode jobs alone and in one batch with other jobs: identical bests."""
    S = 50
    jobs = [(8, 24, 3), (32, 8, 4), (12, 40, 5)]
    sched = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
    betas = orc.schedule(orc.SCHED_GEOMETRIC, 0.1, 5.0, S)
    insts, opts, alone = [], [], []
    try:
        for L, R, seed in jobs:
            J = syn.ea_couplings(L, "pm1", seed)
            inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L)
            insts.append(inst)
            eu, ev, col = orc.ea_graph(L)
            full = orc.anneal_ea(L, J.astype(np.float64), None, betas, R, seed)
            t = float(np.median(full["best_E"]))
            opts.append(pb.make_opts(pb.PB_FORM_RESIDENT, t, pb.PB_FLAG_STOP_AT_TARGET))
            alone.append(_gpu_run(pb, inst, sched, R, seed, pb.PB_FORM_RESIDENT, t))
        bq = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, syn.biclique_couplings(128, "pm1", 2), None, n=128)
        insts.append(bq)
        opts.append(pb.make_opts(pb.PB_FORM_TENSOR))
        import torch
        side = torch.cuda.Stream()
        runs = pb.pb_anneal_batch(insts, [sched] * len(insts), [R for _, R, _ in jobs] + [64],
                                  [seed for _, _, seed in jobs] + [9], opts, stream=side)
        try:
            for q, (L, R, _) in enumerate(jobs):
                fe, be, bs = pb.pb_energy(runs[q], R)
                assert np.array_equal(be, alone[q]["best_E"]) and np.array_equal(bs, alone[q]["best_sweep"])
                assert np.array_equal(pb.pb_best_states(runs[q], R, L ** 3), alone[q]["best_state"])
                assert np.array_equal(pb.pb_target_sweeps(runs[q], R), alone[q]["target_sweep"])
        finally:
            for r in runs:
                pb.pb_run_destroy(r)
    finally:
        for i in insts:
            pb.pb_instance_destroy(i)


@pytest.mark.parametrize("topo,form", [("ea", "resident"), ("bq", "resident")])
def test_stop_ends_the_run_early(pb, topo, form):
    """A target every replica reaches within a few sweeps: the run with 4000 sweeps ends
    far sooner than the same run without the stop (forms that run the whole anneal in one
    launch; the launch-per-sweep forms still issue their remaining launches, which return
    at once)."""
    S, R = 4000, 64
    sched = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 1.0, 3.0)
    if topo == "ea":
        inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(16, "pm1", 3), None, L=16)
        target = 0.0          # E <= 0 is reached within a sweep or two at beta >= 1
    else:
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, syn.biclique_couplings(96, "pm1", 3), None, n=96)
        target = 0.0
    f = pb.PB_FORM_RESIDENT if form == "resident" else pb.PB_FORM_TENSOR
    try:
        pb.pb_run_destroy(pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_LINEAR, 4, 1.0, 3.0), R, 1,
                                       pb.make_opts(f)))  # warm-up
        run = pb.pb_anneal(inst, sched, R, 5, pb.make_opts(f, target))
        t_full = pb.pb_run_device_ms(run)
        pb.pb_run_destroy(run)
        g = _gpu_run(pb, inst, sched, R, 5, f, target)
    finally:
        pb.pb_instance_destroy(inst)
    assert np.all(g["target_sweep"] >= 0) and np.all(g["target_sweep"] < 10)
    assert g["device_ms"] < 0.5 * t_full, (g["device_ms"], t_full)

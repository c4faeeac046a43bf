"""Mixed-topology batches, the autotuner and the request server on the GPU.

Every job of a batch or of the server must give exactly the result of the same
anneal run alone (the runs are deterministic functions of instance, schedule,
replicas and seed), and +-1 jobs also match the CPU oracle bit for bit.
"""
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


# topo, size, law, R, S, kind, b0, b1, hmax, seed, form
JOBS = [
    ("ea", 8, "pm1", 64, 50, 1, 0.1, 5.0, 0, 1, "auto"),
    ("ea", 6, "gauss", 32, 40, 0, 0.1, 3.0, 0, 2, "auto"),
    ("bq", 64, "pm1", 50, 30, 0, 0.35, 3.5, 0, 3, "tensor"),
    ("bq", 40, "gauss", 20, 25, 0, 0.35, 3.5, 0, 4, "cudacore"),
    ("bq", 128, "pm1", 300, 20, 1, 0.1, 5.0, 2, 5, "auto"),
    ("ea", 12, "pm1", 16, 10, 0, 0.1, 3.0, 0, 6, "plain"),
    ("ea", 16, "pm1", 128, 12, 1, 0.1, 5.0, 1, 7, "auto"),
    ("bq", 300, "unif", 40, 8, 0, 0.35, 3.5, 0, 8, "tensor"),
]

FORMS = {"auto": 0, "plain": 1, "resident": 2, "cudacore": 3, "tensor": 4}


def _make(pb, job):
    topo, size, law, R, S, kind, b0, b1, hmax, seed, form = job
    dist = {"pm1": pb.PB_DIST_PM1, "gauss": pb.PB_DIST_GAUSS, "unif": pb.PB_DIST_UNIF}[law]
    if topo == "ea":
        J = pb.pb_generate_ea(size, dist, 100 + seed)
        h = syn.int_fields(size ** 3, hmax, seed) if hmax else None
        inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=size)
    else:
        J = pb.pb_generate_biclique(size, dist, 100 + seed)
        h = syn.int_fields(2 * size, hmax, seed) if hmax else None
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, h, n=size)
    sc = pb.make_schedule(kind, S, b0, b1)
    return inst, sc, R, 1000 + seed, pb.make_opts(FORMS[form])


def _read(pb, run, R, N):
    fe, be, bs = pb.pb_energy(run, R)
    return dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb.pb_final_states(run, R, N),
                best_state=pb.pb_best_states(run, R, N))


def _alone(pb, inst, sc, R, seed, opts):
    run = pb.pb_anneal(inst, sc, R, seed, opts)
    try:
        return _read(pb, run, R, pb.pb_instance_spins(inst))
    finally:
        pb.pb_run_destroy(run)


def _same(a, b):
    for k in ("final_E", "best_E", "best_sweep", "final_state", "best_state"):
        assert np.array_equal(a[k], b[k]), k


def test_mixed_batch_equals_alone(pb):
    made = [_make(pb, j) for j in JOBS]
    try:
        runs = pb.pb_anneal_batch([m[0] for m in made], [m[1] for m in made], [m[2] for m in made],
                                  [m[3] for m in made], [m[4] for m in made])
        try:
            got = [_read(pb, r, m[2], pb.pb_instance_spins(m[0])) for r, m in zip(runs, made)]
        finally:
            for r in runs:
                pb.pb_run_destroy(r)
        for g, m in zip(got, made):
            _same(g, _alone(pb, *m))
    finally:
        for m in made:
            pb.pb_instance_destroy(m[0])


def test_mixed_batch_matches_oracle(pb, orc):
    """+-1 jobs of a mixed batch against the CPU oracle (bit-exact)."""
    jobs = [JOBS[0], JOBS[2], JOBS[4]]
    made = [_make(pb, j) for j in jobs]
    try:
        runs = pb.pb_anneal_batch([m[0] for m in made], [m[1] for m in made], [m[2] for m in made],
                                  [m[3] for m in made], [m[4] for m in made])
        try:
            got = [_read(pb, r, m[2], pb.pb_instance_spins(m[0])) for r, m in zip(runs, made)]
        finally:
            for r in runs:
                pb.pb_run_destroy(r)
    finally:
        for m in made:
            pb.pb_instance_destroy(m[0])
    for job, g in zip(jobs, got):
        topo, size, law, R, S, kind, b0, b1, hmax, seed, form = job
        betas = orc.schedule(kind, b0, b1, S)
        if topo == "ea":
            J = pb.pb_generate_ea(size, pb.PB_DIST_PM1, 100 + seed)
            h = syn.int_fields(size ** 3, hmax, seed) if hmax else None
            o = orc.anneal_ea(size, J.astype(np.float64), None if h is None else h.astype(np.float64), betas, R,
                              1000 + seed)
        else:
            J = pb.pb_generate_biclique(size, pb.PB_DIST_PM1, 100 + seed)
            h = syn.int_fields(2 * size, hmax, seed) if hmax else None
            o = orc.anneal_biclique(size, J.astype(np.float64), None if h is None else h.astype(np.float64), betas,
                                    R, 1000 + seed)
        for k in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
            assert np.array_equal(g[k], o[k]), (job, k)


def test_autotune_records_choice(pb):
    pb.pb_autotune_clear()
    inst, sc, R, seed, _ = _make(pb, JOBS[6])
    try:
        t = pb.pb_autotune(inst, R, 6)
        assert t.n_candidates >= 2
        forms = [t.candidate_form[c] for c in range(t.n_candidates)]
        assert t.form in forms
        assert all(t.probe_ms[c] > 0 for c in range(t.n_candidates))
        if t.form == pb.PB_FORM_RESIDENT:
            assert t.tile_width >= 1
        # a PB_FORM_AUTO anneal now follows the table and still gives the same result
        a = _alone(pb, inst, sc, R, seed, pb.make_opts(pb.PB_FORM_AUTO))
        b = _alone(pb, inst, sc, R, seed, pb.make_opts(pb.PB_FORM_PLAIN))
        _same(a, b)
    finally:
        pb.pb_autotune_clear()
        pb.pb_instance_destroy(inst)
    binst, bsc, bR, bseed, _ = _make(pb, JOBS[2])
    try:
        t = pb.pb_autotune(binst, bR, 4)
        assert t.form in (pb.PB_FORM_TENSOR, pb.PB_FORM_CUDACORE, pb.PB_FORM_RESIDENT) and t.n_candidates == 4
        # the tensor form is tried with whole tiles and with the last round split into half-width tiles
        tensor_wt = sorted(t.candidate_wt[c] for c in range(t.n_candidates) if t.candidate_form[c] == pb.PB_FORM_TENSOR)
        assert tensor_wt == [0, 1]
        # a PB_FORM_AUTO anneal follows the table (form and tile choice) and gives the same result as the
        # explicit tensor form (both tile choices give identical trajectories)
        a = _alone(pb, binst, bsc, bR, bseed, pb.make_opts(pb.PB_FORM_AUTO))
        b = _alone(pb, binst, bsc, bR, bseed, pb.make_opts(pb.PB_FORM_TENSOR))
        _same(a, b)
    finally:
        pb.pb_autotune_clear()
        pb.pb_instance_destroy(binst)


def test_server_results_equal_alone(pb):
    """Jobs submitted together (overlapping on the device) give the alone results."""
    made = [_make(pb, j) for j in JOBS] * 3  # each instance three times, different seeds below
    sv = pb.pb_server_create()
    try:
        tickets = []
        for k, m in enumerate(made):
            tickets.append(pb.pb_server_submit(sv, m[0], m[1], m[2], m[3] + 17 * k, m[4]))
        got = []
        for t, m in zip(tickets, made):
            run, lat = pb.pb_server_wait(sv, t, 120000)
            assert lat > 0
            try:
                got.append(_read(pb, run, m[2], pb.pb_instance_spins(m[0])))
            finally:
                pb.pb_run_destroy(run)
        st = pb.pb_server_stats_get(sv)
        assert st.completed == len(made) and st.failed == 0 and st.queued == 0 and st.inflight == 0
        assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
        for k, (g, m) in enumerate(zip(got, made)):
            _same(g, _alone(pb, m[0], m[1], m[2], m[3] + 17 * k, m[4]))
    finally:
        pb.pb_server_destroy(sv)
        for m in made[: len(JOBS)]:
            pb.pb_instance_destroy(m[0])


def test_server_admission_budget(pb):
    """A device budget of two of the largest jobs: every job still completes, the
    admitted footprint never exceeds the budget, and a job larger than the budget is
    refused at submit."""
    made = [_make(pb, j) for j in JOBS]
    try:
        fp = [pb.pb_run_footprint(m[0], m[1], m[2], m[4]) for m in made]
        assert all(f > 0 for f in fp)
        budget = 2 * max(fp)
        sv = pb.pb_server_create(max_device_bytes=budget, max_inflight=3)
        try:
            tickets = [pb.pb_server_submit(sv, m[0], m[1], m[2], m[3], m[4]) for m in made]
            for t in tickets:
                run, _ = pb.pb_server_wait(sv, t, 120000)
                pb.pb_run_destroy(run)
            st = pb.pb_server_stats_get(sv)
            assert st.completed == len(made)
            assert st.peak_inflight_bytes <= budget
            big = _make(pb, ("bq", 1024, "pm1", 4096, 2, 0, 0.1, 1.0, 0, 9, "tensor"))
            try:
                with pytest.raises(pb.PbError, match="PB_EINVAL"):
                    pb.pb_server_submit(sv, big[0], big[1], big[2], big[3], big[4])
            finally:
                pb.pb_instance_destroy(big[0])
        finally:
            pb.pb_server_destroy(sv)
    finally:
        for m in made:
            pb.pb_instance_destroy(m[0])

"""GPU parity of the biclique K_{n,n} path against the CPU oracle.

+-1 couplings: bit-exact trajectories (integer fields, FP64-built threshold
table).  Real couplings: fields within 1e-5 of FP64 relative to
sum_j |J_ij| + |h_i|, returned-state energies in FP64 within 1e-9 relative,
ensemble mean energy per spin within 3 standard errors.
"""
import math

import numpy as np
import pytest

import synth_inputs as syn

pytestmark = pytest.mark.gpu

FORMS = ["cudacore", "tensor", "resident"]   # anneal forms
FIELD_FORMS = ["cudacore", "tensor"]         # forms with a field entry point


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def _form(pb, name):
    return {"cudacore": pb.PB_FORM_CUDACORE, "tensor": pb.PB_FORM_TENSOR, "resident": pb.PB_FORM_RESIDENT}[name]


def _gpu(pb, n, J, h, sc, R, seed, form):
    return pb.anneal(pb.PB_TOPO_BICLIQUE, J, sc, R, seed, h=h, n=n, form=_form(pb, form))


def _orc(orc, n, J, h, betas, R, seed):
    return orc.anneal_biclique(n, np.asarray(J, np.float64), None if h is None else np.asarray(h, np.float64),
                               betas, R, seed)


CASES = [
    # n, R, S, kind, b0, b1, hmax, seed
    (32, 8, 60, 0, 0.05, 1.0, 0, 1),
    (37, 5, 25, 0, 0.05, 0.8, 0, 2),
    (64, 64, 20, 1, 0.01, 1.0, 0, 3),
    (20, 3, 40, 0, 0.35, 3.5, 2, 4),
    (130, 70, 6, 0, 0.02, 0.3, 0, 5),
    (9, 1, 0, 0, 0.1, 0.1, 0, 6),
    (256, 300, 8, 1, 0.01, 0.2, 0, 7),
    (200, 20, 10, 0, 0.005, 0.1, 3, 8),
]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}R{c[1]}S{c[2]}h{c[6]}" for c in CASES])
def test_pm1_bit_exact(pb, orc, case, form):
    n, R, S, kind, b0, b1, hmax, seed = case
    J = syn.biclique_couplings(n, "pm1", seed)
    h = syn.int_fields(2 * n, hmax, seed + 1) if hmax else None
    sc = pb.make_schedule(kind, S, b0, b1)
    ob = orc.schedule(kind, b0, b1, S)
    g = _gpu(pb, n, J, h, sc, R, seed, form)
    o = _orc(orc, n, J, h, ob, R, seed)
    for k in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[k], o[k]), k


@pytest.mark.parametrize("form", FORMS)
def test_ferromagnet_closed_form(pb, form):
    n = 64
    J = np.ones((n, n), np.int8)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, 100, 0.01, 0.5)
    g = _gpu(pb, n, J, None, sc, 16, 3, form)
    assert np.all(g["best_E"] == -n * n)


@pytest.mark.parametrize("form", FIELD_FORMS)
@pytest.mark.parametrize("n", [96, 300])
def test_f32_fields(pb, orc, form, n):
    J = syn.biclique_couplings(n, "gauss", 11)
    h = syn.real_fields(2 * n, 0.5, 12)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, h, n=n)
    try:
        m = syn.states(5, 2 * n, 13)
        F = pb.pb_fields_ex(inst, m, _form(pb, form))
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, _ = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)
    hd = h.astype(np.float64)
    scale = orc.fields(eu, ev, np.abs(Jd), np.abs(hd), np.ones(2 * n, np.int8))
    for r in range(5):
        F64 = orc.fields(eu, ev, Jd, hd, m[r])
        assert np.all(np.abs(F[r] - F64) <= 1e-5 * scale)


@pytest.mark.parametrize("law", ["gauss", "unif"])
@pytest.mark.parametrize("n", [2048, 4096])
def test_split_bf16_fields_full_size(pb, orc, n, law):
    """Split hi + lo BF16 products with FP32 accumulation in tensor memory (K = n, many
    K stages and tile rounds) against the FP64 field of the same states, at the
    benchmark's sizes: within 1e-5 of sum_j |J_ij| for every spin, on random +-1
    states and on a fully aligned state (all +1)."""
    dist = pb.PB_DIST_GAUSS if law == "gauss" else pb.PB_DIST_UNIF
    J = pb.pb_generate_biclique(n, dist, 17 + n)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n)
    m = np.concatenate([syn.states(3, 2 * n, 19), np.ones((1, 2 * n), np.int8)])
    try:
        F = pb.pb_fields_ex(inst, m, pb.PB_FORM_TENSOR)
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, _ = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)
    scale = orc.fields(eu, ev, np.abs(Jd), None, np.ones(2 * n, np.int8))
    worst = 0.0
    for r in range(m.shape[0]):
        F64 = orc.fields(eu, ev, Jd, None, m[r])
        worst = max(worst, float(np.max(np.abs(F[r] - F64) / scale)))
    assert worst <= 1e-5, worst


@pytest.mark.parametrize("form", FORMS)
def test_f32_energies_and_ensemble(pb, orc, form):
    n, R, S = 48, 128, 80
    J = syn.biclique_couplings(n, "unif", 21)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    ob = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S)
    g = _gpu(pb, n, J, None, sc, R, 5, form)
    eu, ev, _ = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)
    for r in range(R):
        e = orc.energy(eu, ev, Jd, None, g["best_state"][r])
        assert abs(g["best_E"][r] - e) <= 1e-9 * abs(e)
    o = _orc(orc, n, J, None, ob, R, 5)
    eg, eo = g["final_E"] / (2 * n), o["final_E"] / (2 * n)
    se = math.sqrt(eg.var(ddof=1) / R + eo.var(ddof=1) / R)
    assert abs(eg.mean() - eo.mean()) <= 3 * se + 1e-12


@pytest.mark.parametrize("form", FIELD_FORMS)
def test_pm1_fields_exact(pb, orc, form):
    n = 160
    J = syn.biclique_couplings(n, "pm1", 31)
    h = syn.int_fields(2 * n, 4, 32)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, h, n=n)
    try:
        m = syn.states(3, 2 * n, 33)
        F = pb.pb_fields_ex(inst, m, _form(pb, form))
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, _ = orc.biclique_graph(n)
    for r in range(3):
        assert np.array_equal(F[r].astype(np.float64), orc.fields(eu, ev, J.astype(float).reshape(-1), h.astype(float), m[r]))


def test_tensor_multi_tile_ensemble(pb, orc):
    """Split-BF16 tensor form at n = 1024 with 512 replicas (four 256-row tiles per side,
    two replica tiles, persistent rounds) against the oracle's law: final and best energy
    per spin, means within 3 standard errors, two-sample KS p >= 0.001."""
    stats = pytest.importorskip("scipy.stats")
    from concurrent.futures import ThreadPoolExecutor
    n, R, S, R_orc = 1024, 512, 30, 96
    J = pb.pb_generate_biclique(n, pb.PB_DIST_GAUSS, 23)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g = _gpu(pb, n, J, None, sc, R, 29, "tensor")
    ob = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S)
    eu, ev, col = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)

    def part(r0):
        return orc.anneal(eu, ev, Jd, None, col, ob, 6, 29, r_first=r0)

    with ThreadPoolExecutor(max_workers=16) as ex:
        parts = list(ex.map(part, range(0, R_orc, 6)))
    for key in ("final_E", "best_E"):
        eg = g[key] / (2 * n)
        eo = np.concatenate([p[key] for p in parts]) / (2 * n)
        se = math.sqrt(eg.var(ddof=1) / eg.size + eo.var(ddof=1) / eo.size)
        assert abs(eg.mean() - eo.mean()) <= 3 * se, (key, eg.mean(), eo.mean(), se)
        assert float(stats.ks_2samp(eg, eo).pvalue) >= 1e-3, key


def test_tensor_sampled_large(pb, orc):
    """n = 2048, 512 replicas (two replica tiles), 30 sweeps on tensor cores; three
    replicas replayed one by one on the oracle, bit-exact."""
    n, R, S = 2048, 512, 30
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 5)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g = _gpu(pb, n, J, None, sc, R, 9, "tensor")
    ob = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S)
    eu, ev, col = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)
    for r in (0, 257, 511):
        o = orc.anneal(eu, ev, Jd, None, col, ob, 1, 9, r_first=r)
        assert np.array_equal(o["final_state"][0], g["final_state"][r])
        assert o["best_E"][0] == g["best_E"][r] and o["best_sweep"][0] == g["best_sweep"][r]


def test_tensor_full_size_sampled(pb, orc):
    """The biclique bench size and launch configuration: n = 4096, R = 4096 on tensor
    cores (persistent clusters over 16 x 32 pair tiles).  +-1: replicas 0, 2049 and
    4095 replayed one by one on the oracle, bit-exact.  N(0, 1) with the BF16 split:
    the returned best states' energies, recomputed by the oracle in FP64, equal the
    returned best energies within 1e-9 relative, for sampled replicas."""
    n, R, S = 4096, 4096, 4
    eu, ev, col = orc.biclique_graph(n)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    ob = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S)
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 41)
    g = _gpu(pb, n, J, None, sc, R, 43, "tensor")
    Jd = J.astype(np.float64).reshape(-1)
    for r in (0, 2049, 4095):
        o = orc.anneal(eu, ev, Jd, None, col, ob, 1, 43, r_first=r)
        assert np.array_equal(o["final_state"][0], g["final_state"][r])
        assert np.array_equal(o["best_state"][0], g["best_state"][r])
        assert o["best_E"][0] == g["best_E"][r] and o["best_sweep"][0] == g["best_sweep"][r]
    Jg = pb.pb_generate_biclique(n, pb.PB_DIST_GAUSS, 47)
    g = _gpu(pb, n, Jg, None, sc, R, 53, "tensor")
    Jgd = Jg.astype(np.float64).reshape(-1)
    for r in (1, 1500, 4094):
        e = orc.energy(eu, ev, Jgd, None, g["best_state"][r])
        assert abs(g["best_E"][r] - e) <= 1e-9 * abs(e)


@pytest.mark.parametrize("stop", [False, True])
def test_tensor_chained_launches_equal_cudacore(pb, stop):
    """n = 4096 with 1280 replicas: 80 tiles of 256 replicas, at least one per CTA pair, so the
    tensor form chains its sweep loop's launches as programmatic dependents.  +-1 couplings:
    its trajectories equal the FP32 CUDA-core form's bit for bit (both exact), with and
    without the stop rule (a target about half the replicas reach)."""
    n, R, S = 4096, 1280, 6
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 61)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    try:
        out = {}
        for form in (pb.PB_FORM_CUDACORE, pb.PB_FORM_TENSOR):
            target = float("nan")
            if stop:
                run = pb.pb_anneal(inst, sc, R, 63, pb.make_opts(pb.PB_FORM_CUDACORE))
                target = float(np.median(pb.pb_energy(run, R)[1]))
                pb.pb_run_destroy(run)
            opts = pb.make_opts(form, target, pb.PB_FLAG_STOP_AT_TARGET) if stop else pb.make_opts(form)
            run = pb.pb_anneal(inst, sc, R, 63, opts)
            try:
                fe, be, bs = pb.pb_energy(run, R)
                out[form] = dict(fe=fe, be=be, bs=bs, fs=pb.pb_final_states(run, R, 2 * n),
                                 bst=pb.pb_best_states(run, R, 2 * n), ts=pb.pb_target_sweeps(run, R))
            finally:
                pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)
    a, b = out[pb.PB_FORM_CUDACORE], out[pb.PB_FORM_TENSOR]
    for k in ("fe", "be", "bs", "fs", "bst", "ts"):
        assert np.array_equal(a[k], b[k]), k
    if stop:
        assert 0 < (a["ts"] >= 0).sum() < R


def test_tensor_largest_biclique(pb):
    """n = 16384 per side, the largest biclique the library takes, on tensor cores with
    300 replicas (a ragged replica tile): a ferromagnet (J = +1) at beta = 2 from random
    starts reaches one of its two ground states, E0 = -n^2 (all spins aligned), within
    the first two sweeps in every replica.  (Side A aligns with side B's majority; in
    the rare replica whose random side B sums to 0, the second sweep aligns it.)"""
    n, R, S = 16384, 300, 4
    J = np.ones((n, n), np.int8)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 2.0, 2.0)
    g = _gpu(pb, n, J, None, sc, R, 5, "tensor")
    assert np.all(g["best_E"] == -float(n) * n)
    assert np.all(g["best_sweep"] <= 1)
    assert np.all(np.abs(g["best_state"].astype(np.int64).sum(axis=1)) == 2 * n)


def test_tensor_threshold_row_in_global_memory(pb, orc):
    """n = 4300 at small beta: the threshold row (2n + 1 entries) is larger than the
    shared-memory table region and its unsaturated window is wider than 256, so the
    decisions read it from global memory.  Two replicas replayed on the oracle."""
    n, R, S = 4300, 256, 3
    J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 15)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.001, 0.004)
    g = _gpu(pb, n, J, None, sc, R, 19, "tensor")
    ob = orc.schedule(orc.SCHED_LINEAR, 0.001, 0.004, S)
    eu, ev, col = orc.biclique_graph(n)
    Jd = J.astype(np.float64).reshape(-1)
    for r in (0, 255):
        o = orc.anneal(eu, ev, Jd, None, col, ob, 1, 19, r_first=r)
        assert np.array_equal(o["final_state"][0], g["final_state"][r])
        assert o["best_E"][0] == g["best_E"][r] and o["best_sweep"][0] == g["best_sweep"][r]


def test_resident_limits_and_blocks(pb, orc):
    """Resident form: ragged replica counts over several 32-replica CTAs, bit-exact; too
    large an instance is refused."""
    n, R, S = 256, 70, 12
    J = syn.biclique_couplings(n, "pm1", 61)
    h = syn.int_fields(2 * n, 2, 62)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    g = _gpu(pb, n, J, h, sc, R, 63, "resident")
    o = _orc(orc, n, J, h, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), R, 63)
    for k in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(g[k], o[k]), k
    with pytest.raises(pb.PbError, match="PB_EUNSUPPORTED"):
        _gpu(pb, 300, syn.biclique_couplings(300, "pm1", 1), None, sc, 4, 1, "resident")
    with pytest.raises(pb.PbError, match="PB_EUNSUPPORTED"):
        _gpu(pb, 160, syn.biclique_couplings(160, "gauss", 1), None, sc, 4, 1, "resident")

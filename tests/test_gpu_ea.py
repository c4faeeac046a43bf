"""GPU parity of the EA (periodic L^3 cube) path against the CPU oracle.

+-1 instances: bit-exact final/best energies, best sweeps and states (the
decision compares the same Philox word with the same FP64-built threshold).
Gaussian instances: FP32 fields within 1e-5 of FP64 relative to
sum_j |J_ij| + |h_i|; returned-state energies recomputed in FP64 within 1e-9
relative; ensemble mean energy per spin within 3 standard errors.
Inputs come from the neutral seeded module ``synth_inputs``.
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


def _sched(pb, orc, kind, S, b0, b1, d=1, betas=None):
    sc = pb.make_schedule(kind, S, b0, b1, d, betas)
    ob = orc.schedule(kind, b0, b1, S, d, betas)
    return sc, ob


def _gpu(pb, L, J, h, sc, R, seed, form, target=math.nan):
    return pb.anneal(pb.PB_TOPO_EA3D, J, sc, R, seed, h=h, L=L, form=form, target_energy=target)


def _orc(orc, L, J, h, betas, R, seed, **kw):
    return orc.anneal_ea(L, np.asarray(J, np.float64), None if h is None else np.asarray(h, np.float64), betas, R,
                         seed, **kw)


def _assert_same(g, o):
    assert np.array_equal(g["final_state"], o["final_state"])
    assert np.array_equal(g["best_state"], o["best_state"])
    assert np.array_equal(g["final_E"], o["final_E"])
    assert np.array_equal(g["best_E"], o["best_E"])
    assert np.array_equal(g["best_sweep"], o["best_sweep"])


def test_generators_match_oracle(pb, orc):
    for L in (2, 5, 8):
        for dist in (0, 1, 2):
            g = pb.pb_generate_ea(L, dist, 1234 + L)
            o = orc.gen_ea(L, dist, 1234 + L)
            assert np.array_equal(g.astype(np.float64), o)
    for n in (7, 33):
        for dist in (0, 1, 2):
            assert np.array_equal(pb.pb_generate_biclique(n, dist, 99).astype(np.float64), orc.gen_biclique(n, dist, 99))


@pytest.mark.parametrize("form", ["plain", "resident"])
def test_config1_bit_exact(pb, orc, form):
    # EA L=6, +-1 bonds, h=0, checkerboard, linear beta 0.1 -> 3.0, 1000 sweeps, 64 replicas, seed 42
    L, R, S, seed = 6, 64, 1000, 42
    J = syn.ea_couplings(L, "pm1", 1)
    sc, ob = _sched(pb, orc, pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    f = pb.PB_FORM_PLAIN if form == "plain" else pb.PB_FORM_RESIDENT
    g = _gpu(pb, L, J, None, sc, R, seed, f)
    o = _orc(orc, L, J, None, ob, R, seed)
    _assert_same(g, o)


CASES = [
    # L, R, S, kind, b0, b1, d, hmax, seed
    (2, 5, 7, 0, 0.1, 2.0, 1, 0, 3),
    (4, 1, 20, 1, 0.2, 4.0, 1, 0, 4),
    (4, 3, 0, 0, 0.1, 1.0, 1, 0, 5),
    (8, 64, 40, 0, 0.1, 3.0, 3, 0, 6),
    (10, 9, 6, 0, 0.5, 1.5, 1, 0, 7),
    (12, 70, 5, 1, 0.1, 5.0, 1, 0, 8),
    (16, 40, 12, 1, 0.1, 5.0, 1, 0, 9),
    (32, 8, 4, 0, 0.3, 0.9, 1, 0, 10),
    (24, 13, 6, 1, 0.1, 3.0, 1, 0, 14),   # compile-time L = 24 tile (576 of the CTA's threads), ragged replicas
    (4, 8, 30, 0, 0.1, 3.0, 1, 2, 11),
    (6, 6, 20, 0, 0.05, 2.0, 2, 5, 12),
    (8, 12, 15, 1, 0.1, 5.0, 1, 64, 13),
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}R{c[1]}S{c[2]}h{c[7]}" for c in CASES])
@pytest.mark.parametrize("form", ["plain", "resident"])
def test_edge_cases_bit_exact(pb, orc, case, form):
    L, R, S, kind, b0, b1, d, hmax, seed = case
    J = syn.ea_couplings(L, "pm1", seed)
    h = syn.int_fields(L ** 3, hmax, seed + 100) if hmax else None
    sc, ob = _sched(pb, orc, kind, S, b0, b1, d)
    f = pb.PB_FORM_PLAIN if form == "plain" else pb.PB_FORM_RESIDENT
    _assert_same(_gpu(pb, L, J, h, sc, R, seed, f), _orc(orc, L, J, h, ob, R, seed))


def test_explicit_schedule_with_zero_beta(pb, orc):
    L, R = 6, 10
    betas = np.array([0.0, 0.0, 0.5, 3.0, 0.0, 1.0, 2.0, 2.0])
    J = syn.ea_couplings(L, "pm1", 21)
    sc, ob = _sched(pb, orc, pb.PB_SCHED_EXPLICIT, betas.size, 0, 0, 1, betas)
    for f in (pb.PB_FORM_PLAIN, pb.PB_FORM_RESIDENT):
        _assert_same(_gpu(pb, L, J, None, sc, R, 5, f), _orc(orc, L, J, None, ob, R, 5))


def test_target_sweeps(pb, orc):
    L, R, S = 8, 16, 60
    J = syn.ea_couplings(L, "pm1", 31)
    sc, ob = _sched(pb, orc, pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    o = _orc(orc, L, J, None, ob, R, 7, trace=True)
    target = float(np.median(o["best_E"])) + 2.0
    want = np.array([int(np.argmax(tr <= target)) if (tr <= target).any() else -1 for tr in o["trace_E"]])
    for f in (pb.PB_FORM_PLAIN, pb.PB_FORM_RESIDENT):
        g = _gpu(pb, L, J, None, sc, R, 7, f, target=target)
        assert np.array_equal(g["target_sweep"], want)


def test_batch_equals_alone(pb, orc):
    jobs = [
        (8, "pm1", None, 20, 30, 1),
        (6, "pm1", 3, 64, 40, 2),
        (16, "pm1", None, 32, 10, 3),
        (8, "gauss", None, 12, 20, 4),
        (32, "pm1", None, 4, 3, 5),
    ]
    insts, scheds, reps, seeds, alone = [], [], [], [], []
    for L, law, hmax, R, S, seed in jobs:
        J = syn.ea_couplings(L, law, seed)
        h = syn.int_fields(L ** 3, hmax, seed) if hmax else None
        sc = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
        insts.append(pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=L))
        scheds.append(sc); reps.append(R); seeds.append(seed)
        alone.append(_gpu(pb, L, J, h, sc, R, seed, pb.PB_FORM_RESIDENT))
    import torch
    side = torch.cuda.Stream()          # non-default stream: the launch is graph-captured
    runs = pb.pb_anneal_batch(insts, scheds, reps, seeds, stream=side)
    try:
        for q, (L, law, hmax, R, S, seed) in enumerate(jobs):
            N = L ** 3
            fe, be, bs = pb.pb_energy(runs[q], R)
            fs = pb.pb_final_states(runs[q], R, N)
            bst = pb.pb_best_states(runs[q], R, N)
            a = alone[q]
            assert np.array_equal(fs, a["final_state"])
            assert np.array_equal(fe, a["final_E"])
            if law == "pm1":
                assert np.array_equal(bst, a["best_state"])
                assert np.array_equal(bs, a["best_sweep"])
                assert np.array_equal(be, a["best_E"])
    finally:
        for r in runs:
            pb.pb_run_destroy(r)
        for i in insts:
            pb.pb_instance_destroy(i)


# ------------------------------------------------------------------ Gaussian
def test_f32_fields_tolerance(pb, orc):
    L = 8; N = L ** 3
    J = syn.ea_couplings(L, "gauss", 41)
    h = syn.real_fields(N, 0.7, 42)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=L)
    try:
        m = syn.states(6, N, 43)
        F = pb.pb_fields(inst, m)
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, _ = orc.ea_graph(L)
    Jd = J.astype(np.float64).reshape(-1)
    hd = h.astype(np.float64)
    scale = orc.fields(eu, ev, np.abs(Jd), np.abs(hd), np.ones(N, np.int8))  # sum_j |J_ij| + |h_i|
    for r in range(m.shape[0]):
        F64 = orc.fields(eu, ev, Jd, hd, m[r])
        assert np.all(np.abs(F[r].astype(np.float64) - F64) <= 1e-5 * scale)


def test_pm1_fields_exact(pb, orc):
    L = 6; N = L ** 3
    J = syn.ea_couplings(L, "pm1", 51)
    h = syn.int_fields(N, 3, 52)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=L)
    try:
        m = syn.states(3, N, 53)
        F = pb.pb_fields(inst, m)
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, _ = orc.ea_graph(L)
    for r in range(3):
        assert np.array_equal(F[r].astype(np.float64), orc.fields(eu, ev, J.astype(float).reshape(-1), h.astype(float), m[r]))


def test_l24_tile_and_generic_tile_agree(pb):
    """An FP32 L = 24 job runs the compile-time L = 24 tile alone, and the generic tile
    in a batch with an FP32 L = 32 job (whose kernel holds the L = 32 tile instead):
    the same arithmetic and random words, so bit-identical states, energies and best
    sweeps either way."""
    L, R, S, seed = 24, 12, 30, 33
    J = syn.ea_couplings(L, "gauss", 31)
    sc = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
    alone = _gpu(pb, L, J, None, sc, R, seed, pb.PB_FORM_RESIDENT)
    J32 = syn.ea_couplings(32, "gauss", 35)
    insts = [pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L), pb.pb_create_instance(pb.PB_TOPO_EA3D, J32, None, L=32)]
    import torch
    side = torch.cuda.Stream()
    runs = pb.pb_anneal_batch(insts, [sc, pb.make_schedule(pb.PB_SCHED_GEOMETRIC, 5, 0.1, 5.0)], [R, 4], [seed, 37],
                              stream=side)
    try:
        fe, be, bs = pb.pb_energy(runs[0], R)
        assert np.array_equal(pb.pb_final_states(runs[0], R, L ** 3), alone["final_state"])
        assert np.array_equal(pb.pb_best_states(runs[0], R, L ** 3), alone["best_state"])
        assert np.array_equal(fe, alone["final_E"]) and np.array_equal(be, alone["best_E"])
        assert np.array_equal(bs, alone["best_sweep"])
    finally:
        for r in runs:
            pb.pb_run_destroy(r)
        for i in insts:
            pb.pb_instance_destroy(i)


def test_largest_cube(pb, orc):
    """L = 64, the largest cube the library takes (the resident form stops at L = 32, so
    the library's own choice is the plain form), with 5 replicas (a ragged replica
    word): +-1 bit-exact with the oracle; N(0, 1): the returned states' energies,
    recomputed by the oracle in FP64, within 1e-9 relative."""
    L, R, S = 64, 5, 3
    J = syn.ea_couplings(L, "pm1", 21)
    sc, ob = _sched(pb, orc, pb.PB_SCHED_LINEAR, S, 0.3, 2.0)
    _assert_same(_gpu(pb, L, J, None, sc, R, 23, pb.PB_FORM_AUTO), _orc(orc, L, J, None, ob, R, 23))
    Jg = syn.ea_couplings(L, "gauss", 25)
    g = _gpu(pb, L, Jg, None, sc, R, 27, pb.PB_FORM_AUTO)
    eu, ev, _ = orc.ea_graph(L)
    for key_s, key_e in (("final_state", "final_E"), ("best_state", "best_E")):
        for r in range(R):
            e = orc.energy(eu, ev, Jg.astype(np.float64).reshape(-1), None, g[key_s][r])
            assert abs(g[key_e][r] - e) <= 1e-9 * abs(e)


@pytest.mark.parametrize("form", ["plain", "resident"])
def test_f32_energies_fp64(pb, orc, form):
    L, R, S = 8, 16, 100
    J = syn.ea_couplings(L, "gauss", 61)
    h = syn.real_fields(L ** 3, 0.3, 62)
    sc, _ = _sched(pb, orc, pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    f = pb.PB_FORM_PLAIN if form == "plain" else pb.PB_FORM_RESIDENT
    g = _gpu(pb, L, J, h, sc, R, 8, f)
    eu, ev, _ = orc.ea_graph(L)
    for key_s, key_e in (("final_state", "final_E"), ("best_state", "best_E")):
        for r in range(R):
            e = orc.energy(eu, ev, J.astype(np.float64).reshape(-1), h.astype(np.float64), g[key_s][r])
            assert abs(g[key_e][r] - e) <= 1e-9 * abs(e)
    assert np.all(g["best_E"] <= g["final_E"] + 1e-9 * np.abs(g["final_E"]))


def test_f32_plain_equals_resident(pb):
    L, R, S = 8, 16, 50
    J = syn.ea_couplings(L, "gauss", 71)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    a = _gpu(pb, L, J, None, sc, R, 9, pb.PB_FORM_PLAIN)
    b = _gpu(pb, L, J, None, sc, R, 9, pb.PB_FORM_RESIDENT)
    assert np.array_equal(a["final_state"], b["final_state"])
    assert np.array_equal(a["final_E"], b["final_E"])


def test_f32_ensemble_mean_energy(pb, orc):
    # different FP arithmetic -> different trajectories; the laws must agree
    L, R, S = 6, 256, 200
    N = L ** 3
    J = syn.ea_couplings(L, "gauss", 81)
    sc, ob = _sched(pb, orc, pb.PB_SCHED_LINEAR, S, 0.1, 2.0)
    g = _gpu(pb, L, J, None, sc, R, 11, pb.PB_FORM_RESIDENT)
    o = _orc(orc, L, J, None, ob, R, 11)
    eg, eo = g["final_E"] / N, o["final_E"] / N
    se = math.sqrt(eg.var(ddof=1) / R + eo.var(ddof=1) / R)
    assert abs(eg.mean() - eo.mean()) <= 3 * se + 1e-12


# ------------------------------------------------ full size, sampled replicas
def test_full_size_batch_sampled(pb, orc):
    """The benchmark's batch (L=16 and L=32, +-1 and Gaussian, 1024 replicas, 10^4
    geometric sweeps 0.1 -> 5.0, one graph launch of the per-type persistent kernels): sampled replicas are
    replayed one by one on the oracle (bit-exact for +-1); every returned
    energy is checked against the oracle's FP64 energy of the returned state."""
    S, R = 10000, 1024
    specs = [(16, "pm1", 1), (16, "gauss", 2), (32, "pm1", 3), (32, "gauss", 4)]
    insts, Js, scheds = [], [], []
    for L, law, seed in specs:
        J = pb.pb_generate_ea(L, pb.PB_DIST_PM1 if law == "pm1" else pb.PB_DIST_GAUSS, seed)
        Js.append(J)
        insts.append(pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L))
        scheds.append(pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0))
    runs = pb.pb_anneal_batch(insts, scheds, [R] * 4, [100 + q for q in range(4)])
    ob = orc.schedule(orc.SCHED_GEOMETRIC, 0.1, 5.0, S)
    try:
        for q, (L, law, seed) in enumerate(specs):
            N = L ** 3
            fe, be, bs = pb.pb_energy(runs[q], R)
            bst = pb.pb_best_states(runs[q], R, N)
            fst = pb.pb_final_states(runs[q], R, N)
            eu, ev, _ = orc.ea_graph(L)
            Jd = Js[q].astype(np.float64).reshape(-1)
            pick = np.random.default_rng(q).choice(R, size=24, replace=False)
            for r in pick:
                eb = orc.energy(eu, ev, Jd, None, bst[r])
                ef = orc.energy(eu, ev, Jd, None, fst[r])
                assert abs(be[r] - eb) <= 1e-9 * abs(eb) and abs(fe[r] - ef) <= 1e-9 * abs(ef)
            assert np.all(be <= fe + 1e-9 * np.abs(fe))
            assert np.all((bs >= -1) & (bs < S))
            if law == "pm1":
                sample = [0, 1023] if L == 32 else [0, 513, 1023]
                for r in sample:
                    o = orc.anneal_ea(L, Jd, None, ob, 1, 100 + q, r_first=int(r))
                    assert np.array_equal(o["final_state"][0], fst[r])
                    assert np.array_equal(o["best_state"][0], bst[r])
                    assert o["best_E"][0] == be[r] and o["best_sweep"][0] == bs[r]
    finally:
        for r in runs:
            pb.pb_run_destroy(r)
        for i in insts:
            pb.pb_instance_destroy(i)


# ------------------------------------------------------------------- errors
@pytest.mark.parametrize("L,R,hmax,s0", [(8, 64, 0, 23), (6, 20, 0, 1), (16, 48, 0, 40), (10, 9, 2, 11),
                                         (32, 4, 0, 5)])
def test_resume_split_equals_one_run(pb, L, R, hmax, s0):
    """Checkpoint / resume on the resident form (fast and generic tiles, with and
    without fields): sweeps 0..s0-1, then pb_anneal_resume from that run's final state
    and running best, equal one uninterrupted run bit for bit."""
    S, seed = 40, 8
    J = syn.ea_couplings(L, "pm1", 60 + L)
    h = syn.int_fields(L ** 3, hmax, 4) if hmax else None
    betas = np.geomspace(0.1, 5.0, S)
    full = pb.make_schedule(pb.PB_SCHED_EXPLICIT, S, betas=betas)
    first = pb.make_schedule(pb.PB_SCHED_EXPLICIT, s0, betas=betas[:s0])
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=L)
    N = L ** 3
    opts = pb.make_opts(pb.PB_FORM_RESIDENT)

    def read(run):
        fe, be, bs = pb.pb_energy(run, R)
        return dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb.pb_final_states(run, R, N),
                    best_state=pb.pb_best_states(run, R, N))

    runs = []
    try:
        runs.append(pb.pb_anneal(inst, full, R, seed, opts))
        one = read(runs[-1])
        runs.append(pb.pb_anneal(inst, first, R, seed, opts))
        a = read(runs[-1])
        runs.append(pb.pb_anneal_resume(inst, full, R, seed, s0, a["final_state"], a["best_state"], a["best_E"],
                                        a["best_sweep"]))
        b = read(runs[-1])
    finally:
        for r in runs:
            pb.pb_run_destroy(r)
        pb.pb_instance_destroy(inst)
    for key in ("final_state", "best_state", "final_E", "best_E", "best_sweep"):
        assert np.array_equal(b[key], one[key]), key


def test_errors(pb):
    E = pb.PbError
    with pytest.raises(E) as ei:
        pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(3, "pm1", 1), L=3)
    assert ei.value.status == pb.PB_ECOLOUR
    bad = syn.ea_couplings(4, "pm1", 1).copy(); bad[0, 5] = 2
    with pytest.raises(E) as ei:
        pb.pb_create_instance(pb.PB_TOPO_EA3D, bad, L=4)
    assert ei.value.status == pb.PB_EINVAL
    L = 4; N = 64
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    col = ((x + y + z) & 1).transpose(2, 1, 0).reshape(-1)   # index x + L(y + Lz)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(L, "pm1", 1), colour=col, L=L)
    pb.pb_instance_destroy(inst)
    with pytest.raises(E) as ei:
        pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(L, "pm1", 1), colour=1 - col, L=L)
    assert ei.value.status == pb.PB_EUNSUPPORTED
    c2 = col.copy(); c2[0] = 1 - c2[0]
    with pytest.raises(E) as ei:
        pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(L, "pm1", 1), colour=c2, L=L)
    assert ei.value.status == pb.PB_ECOLOUR
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, syn.ea_couplings(L, "pm1", 1), L=L)
    try:
        with pytest.raises(E) as ei:
            pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_LINEAR, 5, 0.1, 1.0), 0, 1)
        assert ei.value.status == pb.PB_EINVAL
        with pytest.raises(E) as ei:
            pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_GEOMETRIC, 5, 0.0, 1.0), 4, 1)
        assert ei.value.status == pb.PB_EINVAL
        with pytest.raises(E) as ei:
            pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_LINEAR, 5, 0.1, 1.0), 4, 1, pb.make_opts(pb.PB_FORM_TENSOR))
        assert ei.value.status == pb.PB_EUNSUPPORTED
        run = pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_LINEAR, 20000, 0.1, 1.0), 64, 1,
                           pb.make_opts(pb.PB_FORM_PLAIN))
        try:
            assert pb.pb_wait(run, 0) in (pb.PB_ETIMEOUT, pb.PB_OK)
            assert pb.pb_wait(run, -1) == pb.PB_OK
            small = np.empty((1, 1), np.int8)
            st = pb.load().pb_best_states(run, small.ctypes.data_as(__import__("ctypes").c_void_p), 1)
            assert st == pb.PB_EINVAL
        finally:
            pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)

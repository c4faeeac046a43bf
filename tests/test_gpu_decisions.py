"""Decision-level parity of the real-coupling (FP32 / split-BF16) paths against the
FP64 oracle, plus ensemble checks of the fast EA tiles.

Real couplings cannot give bit-exact trajectories (the GPU rounds fields in FP32
or accumulates split BF16 products; the oracle works in FP64), but every single
decision can still be replayed: a run of s0 sweeps and a run of s0 + 1 sweeps
(the same schedule's prefixes, same seed) give the states before and after sweep
s0.  Colour class c of sweep s0 sees classes < c as they are after the sweep and
classes >= c as they were before it (Sec. 1.2.2: update groups in order, no edge
inside a group), so the oracle's one-class step (Eq. 3 field in FP64, Eq. 2
decision with the same Philox word) is run on exactly the neighbour states the
GPU used.  A GPU decision may then differ from the oracle's only where the random
word lies within rounding distance of the p-bit probability:
|w 2^-32 - P| <= 2e-5 (the GPU rule reads the word's top 23 bits, 2^-23, and its
FP32 field and exp2 shift P by well under 1e-5).  Every differing decision must
satisfy that, and there may be at most 1e-5 of them -- a dropped or wrong
coupling term, a wrong beta, sweep or replica index, or a wrong comparison would
break thousands of decisions.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth_inputs as syn

pytestmark = pytest.mark.gpu

EXPLAIN = 2e-5        # |w 2^-32 - P| below which FP32 vs FP64 rounding can flip a decision
MAX_FRAC = 1e-5       # at most this fraction of decisions may differ


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def _prefix_states(pb, inst, betas, s0, R, seed, form, N):
    """GPU states after sweeps 0..s0-1 and 0..s0 (two runs of the schedule's prefixes)."""
    out = []
    for S in (s0, s0 + 1):
        sc = pb.make_schedule(pb.PB_SCHED_EXPLICIT, S, betas=np.ascontiguousarray(betas[:S]))
        run = pb.pb_anneal(inst, sc, R, seed, pb.make_opts(form))
        try:
            out.append(pb.pb_final_states(run, R, N))
        finally:
            pb.pb_run_destroy(run)
    return out


def _chunks(R, picks):
    """Contiguous replica ranges (r_first, count) to replay."""
    if picks is None:
        return [(0, R)]
    return picks


def _replay(orc, eu, ev, J, h, col, betas, s0, before, after, seed, picks):
    """Replay every class of sweep s0 on the oracle from the GPU's own neighbour states;
    returns (decisions, mismatches, unexplained)."""
    k = int(col.max()) + 1
    beta = float(betas[s0])
    tasks = []
    for r0, cnt in _chunks(before.shape[0], picks):
        for c in range(k):
            mixed = np.where(col[None, :] < c, after[r0:r0 + cnt], before[r0:r0 + cnt]).astype(np.int8)
            tasks.append((r0, cnt, c, mixed))

    def one(t):
        r0, cnt, c, mixed = t
        res = orc.class_step(eu, ev, J, h, col, c, beta, s0, mixed, seed, r_first=r0, n_colours=k)
        cls = col == c
        got = after[r0:r0 + cnt][:, cls]
        want = res["state"][:, cls]
        bad = got != want
        u = res["w"][:, cls].astype(np.float64) / 2.0 ** 32
        far = np.abs(u - res["P"][:, cls]) > EXPLAIN
        return int(cls.sum()) * cnt, int(bad.sum()), int((bad & far).sum())

    with ThreadPoolExecutor(max_workers=16) as ex:   # the oracle's C calls release the GIL
        res = list(ex.map(one, tasks))
    return tuple(int(sum(v)) for v in zip(*res))


def _check(n_dec, n_bad, n_unexplained):
    assert n_dec > 0
    assert n_unexplained == 0, (n_dec, n_bad, n_unexplained)
    assert n_bad <= MAX_FRAC * n_dec, (n_dec, n_bad)


GEO = (0.1, 5.0, 100)   # the benchmark's geometric schedule shape, shortened


# EA cubes: (L, R, form, with field, picks).  L = 32 (any R) and L = 16 with R >= 2420 reach the
# compile-time fast tiles (WT = 1 / WT = 4) of the resident form -- the benchmark's Gaussian tiles.
EA_CASES = [
    (32, 256, "resident", False, None),
    (32, 64, "resident", True, None),
    (16, 2432, "resident", False, [(0, 96), (1200, 96), (2336, 96)]),
    (16, 2432, "resident", True, [(0, 64), (2368, 64)]),
    (24, 40, "resident", False, None),      # generic tile, compile-time shape L = 24, WT = 1
    (12, 64, "resident", True, None),       # generic tile, compile-time shape L = 12, WT = 4, with fields
    (10, 32, "resident", False, None),      # generic tile of runtime shape
    (8, 24, "plain", True, None),           # plain form
]


@pytest.mark.parametrize("case", EA_CASES, ids=[f"L{c[0]}R{c[1]}{c[2]}{'h' if c[3] else ''}" for c in EA_CASES])
@pytest.mark.parametrize("s0", [0, 37])
def test_ea_f32_decisions_replayed(pb, orc, case, s0):
    L, R, form, with_h, picks = case
    N = L ** 3
    J = syn.ea_couplings(L, "gauss", 500 + L)
    h = syn.real_fields(N, 0.5, 600 + L) if with_h else None
    betas = orc.schedule(orc.SCHED_GEOMETRIC, *GEO)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, h, L=L)
    f = pb.PB_FORM_RESIDENT if form == "resident" else pb.PB_FORM_PLAIN
    try:
        before, after = _prefix_states(pb, inst, betas, s0, R, 77, f, N)
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, col = orc.ea_graph(L)
    hd = None if h is None else h.astype(np.float64)
    _check(*_replay(orc, eu, ev, J.astype(np.float64).reshape(-1), hd, col, betas, s0, before, after, 77, picks))


# Bicliques: (n, R, law, form, picks).  n = 4096, R = 4096 is the benchmark's tensor-core
# configuration (persistent clusters, several tile rounds), replayed on sampled replicas.
BQ_CASES = [
    (4096, 4096, "gauss", "tensor", [(0, 2), (2049, 2), (4094, 2)]),
    (2048, 512, "unif", "tensor", [(0, 4), (509, 3)]),
    (1024, 1024, "gauss", "tensor", [(0, 8), (1000, 8)]),
    (300, 70, "gauss", "tensor", None),
    (1024, 256, "gauss", "cudacore", [(0, 8), (250, 6)]),
    (96, 40, "unif", "resident", None),
]


@pytest.mark.parametrize("case", BQ_CASES, ids=[f"n{c[0]}R{c[1]}{c[2]}{c[3]}" for c in BQ_CASES])
def test_biclique_real_decisions_replayed(pb, orc, case):
    n, R, law, form, picks = case
    s0 = 9
    J = pb.pb_generate_biclique(n, pb.PB_DIST_GAUSS if law == "gauss" else pb.PB_DIST_UNIF, 31 + n)
    betas = orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, 40)
    inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n)
    f = {"tensor": pb.PB_FORM_TENSOR, "cudacore": pb.PB_FORM_CUDACORE, "resident": pb.PB_FORM_RESIDENT}[form]
    try:
        before, after = _prefix_states(pb, inst, betas, s0, R, 91, f, 2 * n)
    finally:
        pb.pb_instance_destroy(inst)
    eu, ev, col = orc.biclique_graph(n)
    _check(*_replay(orc, eu, ev, J.astype(np.float64).reshape(-1), None, col, betas, s0, before, after, 91, picks))


def test_graph_real_decisions_replayed(pb, orc):
    """General graph (odd periodic cube L = 7: not bipartite, greedy colouring), N(0,1)
    couplings and fields: every class of the sweep replayed."""
    L, R, s0 = 7, 64, 12
    eu, ev = syn.graph_periodic_cube(L)
    N = L ** 3
    J = syn.edge_couplings(eu.size, "gauss", 5)
    h = syn.real_fields(N, 0.3, 6)
    col, k = pb.pb_greedy_colouring(N, eu, ev)
    assert k >= 3
    betas = orc.schedule(orc.SCHED_LINEAR, 0.1, 3.0, 30)
    inst = pb.pb_create_graph_instance(N, eu, ev, J, h, col)
    try:
        before, after = _prefix_states(pb, inst, betas, s0, R, 13, pb.PB_FORM_AUTO, N)
    finally:
        pb.pb_instance_destroy(inst)
    _check(*_replay(orc, eu, ev, J.astype(np.float64), h.astype(np.float64), np.asarray(col, np.int32), betas, s0,
                    before, after, 13, None))


# ----------------------------------------------------- ensembles of the fast tiles
def _ks_p(a, b):
    stats = pytest.importorskip("scipy.stats")
    return float(stats.ks_2samp(a, b).pvalue)


@pytest.mark.parametrize("L,R_gpu,R_orc", [(32, 256, 128), (16, 2432, 256)])
def test_ea_f32_fast_tile_ensemble(pb, orc, L, R_gpu, R_orc):
    """The benchmark's Gaussian fast tiles (L = 32, WT = 1; L = 16, WT = 4) against the
    oracle's law: energy per spin after 25, 50 and 100 sweeps of the geometric schedule
    0.1 -> 5.0: means within 3 standard errors and a two-sample KS test (p >= 0.001)."""
    N = L ** 3
    J = syn.ea_couplings(L, "gauss", 700 + L)
    betas = orc.schedule(orc.SCHED_GEOMETRIC, *GEO)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L)
    gE = {}
    try:
        for S in (25, 50, 100):
            sc = pb.make_schedule(pb.PB_SCHED_EXPLICIT, S, betas=np.ascontiguousarray(betas[:S]))
            run = pb.pb_anneal(inst, sc, R_gpu, 3, pb.make_opts(pb.PB_FORM_RESIDENT))
            try:
                gE[S] = pb.pb_energy(run, R_gpu)[0] / N
            finally:
                pb.pb_run_destroy(run)
    finally:
        pb.pb_instance_destroy(inst)
    Jd = J.astype(np.float64).reshape(-1)
    chunk = max(1, R_orc // 16)

    def orc_part(r0):
        return orc.anneal_ea(L, Jd, None, betas, chunk, 3, r_first=r0, trace=True)["trace_E"]

    with ThreadPoolExecutor(max_workers=16) as ex:
        tr = np.concatenate(list(ex.map(orc_part, range(0, R_orc, chunk))))
    for S in (25, 50, 100):
        eg, eo = gE[S], tr[:, S - 1] / N
        se = math.sqrt(eg.var(ddof=1) / eg.size + eo.var(ddof=1) / eo.size)
        assert abs(eg.mean() - eo.mean()) <= 3 * se, (S, eg.mean(), eo.mean(), se)
        assert _ks_p(eg, eo) >= 1e-3, S

"""Benchmark of the graph-coloured parallel p-bit annealer on GB300.

Workload (one step = one pass of the whole hot path over one batch): the
batched 3D Edwards-Anderson anneal -- cubes L=16 and L=32, +-1 (int8) and
Gaussian N(0,1) (FP32) couplings, h = 0, 1024 replicas each, 10^4 sweeps of a
geometric beta schedule 0.1 -> 5.0, all four jobs in one graph-captured
launch (one persistent kernel per coupling type, the second a programmatic
dependent of the first).  Metric: p-bit updates per second (N * S * R summed
over the jobs, divided by the step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (each rank anneals its own copy of the batch; no
collective on the data path), weak scaling, value = all ranks' updates / max
time over ranks.  The reference arm times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Batches and the request server run many graph-captured anneals on the library's
# launch streams at once: give the process more hardware work queues than the
# default 8 so that independent streams do not share one (set before CUDA starts).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "p-bit updates/s"
UNIT = "updates/s"
S_SWEEPS = 10000
R_REPLICAS = 1024
BETA0, BETA1 = 0.1, 5.0
JOBS = [(16, "pm1", 1), (16, "gauss", 2), (32, "pm1", 3), (32, "gauss", 4)]  # (L, law, instance seed)
CONFIG = {
    "workload": "batched EA: L=16 and L=32 periodic cubes, +-1 (int8) and N(0,1) (FP32) couplings, h=0, "
                "1024 replicas each, 1e4-sweep geometric beta 0.1->5.0, one graph-captured launch: a persistent "
                "kernel per coupling type, chained by programmatic dependent launch",
    "instances": [f"L{L}-{law}-seed{s}" for L, law, s in JOBS],
    "replicas": R_REPLICAS, "sweeps": S_SWEEPS, "schedule": "geometric 0.1->5.0",
    "l2": "L2 flushed (256 MiB write) before every timed step",
}


def profiled_traffic():
    """DRAM bytes of the resident kernels of one bench step, from the committed ncu
    summary, if the kernel sources are unchanged since that capture (else None)."""
    import glob
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2510_23419_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in ("ea.cu", "ea_fast.cuh", "ea_kernels.cuh", "ea_launch.h", "pb_common.h")]
    try:
        h = hashlib.sha256()
        for f in files:
            with open(f, "rb") as fh:
                h.update(fh.read())
        with open(os.path.join(ROOT, "profiles", "ea_resident_batch_dram.md")) as fh:
            txt = fh.read()
    except OSError:
        return None
    stamp = re.search(r"first 16 hex digits\): `([0-9a-f]{16})`", txt)
    val = re.search(r"traffic_bytes_per_launch: (\d+)", txt)
    if not stamp or not val or stamp.group(1) != h.hexdigest()[:16]:
        return None
    return int(val.group(1))


def rank_seeds(rank: int):
    """Replicas only: every rank anneals its own copy of the batch with its own seeds."""
    return [1000 * rank + 100 + q for q in range(len(JOBS))]


def aggregate_ranks(local_ms: float, local_updates: int, dist=None, device="cpu"):
    """Whole-job result over ranks: the slowest rank's time and the sum of all ranks' updates.
    With no process group this is the local result."""
    if dist is None:
        return local_ms, local_updates
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def updates_per_step():
    return sum((L ** 3) * S_SWEEPS * R_REPLICAS for L, _, _ in JOBS)


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        t0 = time.time()  # let the sampler start up before the timed region
        while not self.lines and time.time() - t0 < 5.0:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def oracle_sample(sweeps: int):
    """Time the CPU oracle (as it stands, single-threaded) on replica 0 of each
    job for the first `sweeps` sweeps of the same schedule; instances come from
    the oracle's own generator (same seeds, same couplings as the library's)."""
    from oracle import oracle as orc
    betas = orc.schedule(orc.SCHED_GEOMETRIC, BETA0, BETA1, S_SWEEPS)[:sweeps]
    insts = [(L, orc.gen_ea(L, orc.DIST_PM1 if law == "pm1" else orc.DIST_GAUSS, seed)) for L, law, seed in JOBS]
    t0 = time.perf_counter()
    for L, J in insts:
        orc.anneal_ea(L, J, None, betas, 1, 100)
    dt = time.perf_counter() - t0
    upd = sum(L ** 3 * sweeps for L, _ in insts)
    return upd, dt


def oracle_config1():
    """The CPU oracle on the whole small-cube run shape (EA L = 6, +-1 bonds from seed 1,
    h = 0, linear beta 0.1 -> 3.0, 1000 sweeps, 64 replicas, seed 42), single-threaded,
    as it stands; returns (updates, seconds)."""
    from oracle import oracle as orc
    L, R, S = 6, 64, 1000
    J = orc.gen_ea(L, orc.DIST_PM1, 1)
    betas = orc.schedule(orc.SCHED_LINEAR, 0.1, 3.0, S)
    t0 = time.perf_counter()
    orc.anneal_ea(L, J, None, betas, R, 42)
    return L ** 3 * R * S, time.perf_counter() - t0


def _oracle_replica(task):
    """One host core's share of the all-cores CPU baseline: replica r of each job
    for the first `sweeps` sweeps (the oracle as it stands, single-threaded)."""
    sweeps, r = task
    if r < 0:
        return 0, 0.0  # pool warm-up
    from oracle import oracle as orc
    betas = orc.schedule(orc.SCHED_GEOMETRIC, BETA0, BETA1, S_SWEEPS)[:sweeps]
    insts = [(L, orc.gen_ea(L, orc.DIST_PM1 if law == "pm1" else orc.DIST_GAUSS, seed)) for L, law, seed in JOBS]
    t0 = time.perf_counter()
    for L, J in insts:
        orc.anneal_ea(L, J, None, betas, 1, 100, r_first=r)
    return sum(L ** 3 * sweeps for L, _ in insts), time.perf_counter() - t0


def oracle_sample_all_cores(sweeps: int, cores: int):
    """The same sample spread over `cores` processes (spawned: no CUDA state is
    inherited), replica r in process r; returns (updates, wall seconds of the
    concurrent runs)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_replica, [(0, -1)] * cores)  # start and import in every process first
        t0 = time.perf_counter()
        res = pool.map(_oracle_replica, [(sweeps, r) for r in range(cores)], chunksize=1)
        wall = time.perf_counter() - t0
    return sum(u for u, _ in res), wall


def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    sweeps = 300
    for _ in range(args.warmup):
        oracle_sample(sweeps)
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        u, t = oracle_sample(sweeps)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": CONFIG,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"replica 0 of each of the 4 jobs, first {sweeps} sweeps of the schedule, per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- measured peaks
def measure_dense_peaks(n: int = 8192, reps: int = 10):
    """Dense tensor peaks of this GPU, measured the way the BF16 figure of the
    driver's peak file is: n^3 products, best of `reps`, CUDA events.  FP8 e4m3 with
    torch._scaled_mm (per-tensor unit scales, BF16 output); BF16 with torch.matmul.
    TFLOP/s = 2 n^3 / time."""
    import torch
    out = {"n": n, "reps": reps}

    def best_of(fn):
        fn()
        torch.cuda.synchronize()
        best = math.inf
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return 2.0 * n ** 3 / (best / 1e3) / 1e12

    g = torch.Generator(device="cuda").manual_seed(0)
    a16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16, generator=g)
    b16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16, generator=g)
    out["bf16_tflops"] = best_of(lambda: torch.matmul(a16, b16))
    try:
        a8 = a16.to(torch.float8_e4m3fn)
        b8 = b16.t().contiguous().to(torch.float8_e4m3fn).t()   # column-major second operand
        one = torch.ones((), device="cuda", dtype=torch.float32)
        out["fp8_tflops"] = best_of(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one,
                                                             out_dtype=torch.bfloat16))
        out["fp8_how"] = "torch._scaled_mm e4m3 x e4m3 -> bf16, unit per-tensor scales"
    except Exception as e:  # noqa: BLE001 -- report why, keep the bench going
        out["fp8_tflops"] = None
        out["fp8_error"] = str(e)[:200]
    del a16, b16
    torch.cuda.empty_cache()
    return out


def philox_ceiling(pb, stream, sweeps: int = 200):
    """Measured random-word ceiling of the EA update (one Philox4x32-10 word per update,
    same counters as the resident tiles, nothing else): updates/s, best of 3."""
    best = 0.0
    for _ in range(3):
        ms, upd = pb.pb_philox_ceiling(sweeps, 0, stream=stream)
        best = max(best, upd / (ms / 1e3))
    return best


# ------------------------------------------------------------ biclique
def split_field_error(pb, stream, n: int = 4096, states: int = 4):
    """Error of the split hi + lo BF16 tensor-core field against FP64 (numpy) on the
    bench's biclique size: N(0,1) and U(-1,1) couplings, random +-1 states and the
    all-+1 state; |F - F64| relative to sum_j |J_ij| (max and mean over spins)."""
    import synth_inputs as syn
    out = {"n": n, "states": states, "unit": "|F_tensor - F_fp64| / sum_j |J_ij|"}
    for law, dist in (("gauss", pb.PB_DIST_GAUSS), ("unif", pb.PB_DIST_UNIF)):
        J = pb.pb_generate_biclique(n, dist, 11)
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n, stream=stream)
        m = np.concatenate([syn.states(states - 1, 2 * n, 5), np.ones((1, 2 * n), np.int8)])
        F = pb.pb_fields_ex(inst, m, pb.PB_FORM_TENSOR, stream=stream).astype(np.float64)
        pb.pb_instance_destroy(inst)
        Jd = J.astype(np.float64)
        A = np.abs(Jd)
        scale = np.concatenate([A.sum(axis=1), A.sum(axis=0)])
        mf = m.astype(np.float64)
        F64 = np.concatenate([mf[:, n:] @ Jd.T, mf[:, :n] @ Jd], axis=1)   # left: J m_right, right: J^T m_left
        rel = np.abs(F - F64) / scale
        out[law] = {"max": float(rel.max()), "mean": float(rel.mean()),
                    "bound_per_coupling": 2.0 ** -16}
    return out


def biclique_block(pb, stream, peaks):
    """Biclique K_{n,n}, n = 4096, 4096 replicas, linear beta 0.35 -> 3.5: sweep-loop kernels of the
    tensor-core form (+-1 in FP8 e4m3, N(0,1) in split BF16) and of the FP32 CUDA-core form, timed with
    the library's events around the sweep loop.  Tensor roofline: 2n FLOP per update (e4m3) or 4n
    (two BF16 products) against the measured BF16 peak (x2 for FP8, the nominal dense ratio)."""
    n, R = 4096, 4096
    bf16 = float(peaks.get("bf16_tflops", 1888.9))
    fp8 = peaks.get("fp8_tflops_measured")
    out = {"workload": "biclique n=4096 (8192 spins), 4096 replicas, linear beta 0.35->3.5, h=0"}
    for law, form, S in (("pm1", "tensor", 200), ("gauss", "tensor", 100), ("pm1", "cudacore", 4)):
        J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1 if law == "pm1" else pb.PB_DIST_GAUSS, 11)
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n, stream=stream)
        sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
        f = pb.PB_FORM_TENSOR if form == "tensor" else pb.PB_FORM_CUDACORE
        run = pb.pb_anneal(inst, sc, R, 5, pb.make_opts(f), stream=stream)
        ms = pb.pb_run_kernel_ms(run)
        pb.pb_run_destroy(run)
        pb.pb_instance_destroy(inst)
        upd = 2 * n * R * S
        flop_per_upd = (2 * n) if (law == "pm1" or form == "cudacore") else (4 * n)
        tf = upd * flop_per_upd / (ms / 1e3) / 1e12
        key = f"{law}_{form}"
        ent = {"sweeps": S, "ms": ms, "updates_per_s": upd / (ms / 1e3), "tflops": tf}
        if form == "tensor":
            if law == "pm1":
                peak = fp8 if fp8 else 2 * bf16
                src = ("measured fp8 dense (torch._scaled_mm e4m3, 8192^3, best of 10, this run)" if fp8
                       else "measured bf16 burst x 2 (nominal fp8/bf16 ratio; fp8 measurement failed)")
            else:
                peak, src = bf16, "measured bf16 burst (peak file)"
                # the method's own work is 2n FLOP per update; the split issues 4n
                ent["method_tflops_2n"] = upd * 2 * n / (ms / 1e3) / 1e12
                ent["method_frac_2n"] = ent["method_tflops_2n"] / peak
            ent.update({"peak_tflops": peak, "frac": tf / peak, "peak_source": src})
        out[key] = ent
    out["split_bf16_field_error"] = split_field_error(pb, stream)
    return out


def biclique_sweep_block(pb, stream, peaks):
    """Config 3 over its range: n in {512, 1024, 2048, 4096} x R in {256, 1024, 4096}, linear beta
    0.35 -> 3.5, h = 0; tensor form with +-1 couplings (FP8 e4m3) and N(0,1) (split BF16), and
    the FP32 CUDA-core form (+-1).  Timed with the library's events around the sweep loop;
    FLOP/s on the method's 2n FLOP per update against the measured FP8 / BF16 dense peaks."""
    fp8 = peaks.get("fp8_tflops_measured") or 2 * float(peaks.get("bf16_tflops", 1888.9))
    bf16 = float(peaks.get("bf16_tflops", 1888.9))
    insts = {}
    rows = []
    for n in (512, 1024, 2048, 4096):
        for law in ("pm1", "gauss"):
            J = pb.pb_generate_biclique(n, pb.PB_DIST_PM1 if law == "pm1" else pb.PB_DIST_GAUSS, 13)
            insts[(n, law)] = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=n, stream=stream)
        for R in (256, 1024, 4096):
            for law, form in (("pm1", "tensor"), ("gauss", "tensor"), ("pm1", "cudacore")):
                budget = 4e10 if form == "tensor" else 2e9
                S = int(max(4, min(400, budget / (2 * n * R)))) & ~1
                sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
                f = pb.PB_FORM_TENSOR if form == "tensor" else pb.PB_FORM_CUDACORE
                run = pb.pb_anneal(insts[(n, law)], sc, R, 3, pb.make_opts(f), stream=stream)
                ms = pb.pb_run_kernel_ms(run)
                pb.pb_run_destroy(run)
                ups = 2 * n * R * S / (ms / 1e3)
                tf = ups * 2 * n / 1e12
                peak = fp8 if (form == "tensor" and law == "pm1") else bf16
                rows.append({"n": n, "R": R, "law": law, "form": form, "sweeps": S, "ms": ms, "updates_per_s": ups,
                             "tflops_2n": tf, "frac_2n": tf / peak if form == "tensor" else None,
                             "peak": ("fp8" if law == "pm1" else "bf16") if form == "tensor" else None})
    for i in insts.values():
        pb.pb_instance_destroy(i)
    return {"workload": "biclique K_{n,n}, n in {512,1024,2048,4096}, R in {256,1024,4096}, linear 0.35->3.5, h=0",
            "peaks_tflops": {"fp8": fp8, "bf16": bf16}, "rows": rows}


# ------------------------------------------------------------ config 1
def config1_block(pb, stream):
    """The paper's small-cube run shape (Sec. 2): EA L = 6 (216 spins), +-1 bonds from seed 1,
    h = 0, linear beta 0.1 -> 3.0 over 1000 sweeps, 64 replicas, seed 42.  Latency of one
    whole anneal (create excluded; readout of energies included) in the plain form the
    configuration names, and in the resident form; median of 5 after one warm-up."""
    import torch
    L, R, S = 6, 64, 1000
    J = pb.pb_generate_ea(L, pb.PB_DIST_PM1, 1)
    inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L, stream=stream)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    out = {"workload": "EA L=6 +-J (seed 1), h=0, linear beta 0.1->3.0, 1000 sweeps, 64 replicas, seed 42",
           "updates": L ** 3 * R * S}
    for name, form in (("plain", pb.PB_FORM_PLAIN), ("resident", pb.PB_FORM_RESIDENT)):
        ts = []
        for it in range(6):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run = pb.pb_anneal(inst, sc, R, 42, pb.make_opts(form), stream=stream)
            pb.pb_energy(run, R)
            e1.record(stream)
            e1.synchronize()
            pb.pb_run_destroy(run)
            if it:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[name] = {"ms": ms, "updates_per_s": L ** 3 * R * S / (ms / 1e3)}
    pb.pb_instance_destroy(inst)
    return out


# ------------------------------------------------------ mixed batch, served
def mixed_jobs(count: int, seed: int, s_lo: float, s_hi: float):
    """Jobs of the mixed workload: half EA cubes L in {8,12,16,24}, half bicliques
    n in {128,...,2048}; half +-1, half N(0,1); replicas 2^5..2^10 and sweep budgets
    log-uniform; geometric beta 0.1 -> 5.0."""
    rng = np.random.default_rng(seed)
    jobs = []
    for q in range(count):
        topo = "ea" if rng.random() < 0.5 else "bq"
        size = int(rng.choice([8, 12, 16, 24])) if topo == "ea" else int(rng.choice([128, 256, 512, 1024, 2048]))
        law = "pm1" if rng.random() < 0.5 else "gauss"
        R = int(2 ** rng.integers(5, 11))
        S = int(round(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        jobs.append((topo, size, law, R, S, 7000 + q))
    return jobs


def job_updates(j):
    topo, size, law, R, S, _ = j
    return (size ** 3 if topo == "ea" else 2 * size) * R * S


def make_instances(pb, jobs, stream):
    cache = {}
    insts = []
    for topo, size, law, R, S, iseed in jobs:
        key = (topo, size, law, iseed)
        if key not in cache:
            dist = pb.PB_DIST_PM1 if law == "pm1" else pb.PB_DIST_GAUSS
            if topo == "ea":
                cache[key] = pb.pb_create_instance(pb.PB_TOPO_EA3D, pb.pb_generate_ea(size, dist, iseed), None,
                                                   L=size, stream=stream)
            else:
                cache[key] = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, pb.pb_generate_biclique(size, dist, iseed),
                                                   None, n=size, stream=stream)
        insts.append(cache[key])
    return insts, list(cache.values())


def ks_2samp_p(a, b):
    """p-value of the two-sample Kolmogorov-Smirnov test of two best-energy samples
    (None when scipy is missing or a sample has fewer than two values)."""
    try:
        from scipy import stats
    except ImportError:
        return None
    if np.asarray(a).size < 2 or np.asarray(b).size < 2:
        return None
    return float(stats.ks_2samp(np.asarray(a, np.float64), np.asarray(b, np.float64)).pvalue)


def ks_summary(ps):
    ps = [p for p in ps if p is not None]
    if not ps:
        return {"jobs": 0}
    return {"jobs": len(ps), "p_at_least_0.01": sum(int(p >= 0.01) for p in ps), "min_p": min(ps),
            "median_p": float(np.median(ps))}


def mixed_block(pb, stream):
    """200 mixed instances in one batch (EA jobs in one persistent graph-captured launch,
    bicliques as graph-captured anneals side by side), forms from the autotuner; against
    the plain per-instance forms (EA plain, biclique CUDA-core) run one after another on
    every 4th job."""
    import torch
    jobs = mixed_jobs(200, 7, 500, 1e4)
    insts, owned = make_instances(pb, jobs, stream)
    scheds = [pb.make_schedule(pb.PB_SCHED_GEOMETRIC, j[4], BETA0, BETA1) for j in jobs]
    seeds = [50000 + q for q in range(len(jobs))]
    reps = [j[3] for j in jobs]
    # autotuner: one probe per distinct shape (untimed)
    t0 = time.perf_counter()
    tuned = {}
    for j, i in zip(jobs, insts):
        key = (j[0], j[1], j[2], int(math.ceil(math.log2(j[3]))))
        if key not in tuned:
            t = pb.pb_autotune(i, j[3], 8, stream=stream)
            tuned[key] = (t.form, t.tile_width)
    tune_s = time.perf_counter() - t0

    def timed_batch(idx):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        runs = pb.pb_anneal_batch([insts[q] for q in idx], [scheds[q] for q in idx], [reps[q] for q in idx],
                                  [seeds[q] for q in idx], stream=stream)
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - w0
        best = [pb.pb_energy(r, reps[q])[1] for r, q in zip(runs, idx)]
        for r in runs:
            pb.pb_run_destroy(r)
        return e0.elapsed_time(e1), wall, best

    allq = list(range(len(jobs)))
    timed_batch(allq)  # warm-up (graphs, pools)
    ms, wall, _ = timed_batch(allq)
    upd = sum(job_updates(j) for j in jobs)
    sub = allq[::4]
    sub_upd = sum(job_updates(jobs[q]) for q in sub)
    sms, _, sbest = timed_batch(sub)
    # plain per-instance forms, one job after another
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pruns = []
    for q in sub:
        f = pb.PB_FORM_PLAIN if jobs[q][0] == "ea" else pb.PB_FORM_CUDACORE
        pruns.append(pb.pb_anneal(insts[q], scheds[q], reps[q], seeds[q], pb.make_opts(f), stream=stream))
    e1.record(stream)
    e1.synchronize()
    pms = e0.elapsed_time(e1)
    pbest = [pb.pb_energy(r, reps[q])[1] for r, q in zip(pruns, sub)]
    for r in pruns:
        pb.pb_run_destroy(r)
    # +-1 jobs: the same trajectories bit for bit; N(0,1) jobs (split BF16 tensor
    # products vs FP32 CUDA-core fields round differently): mean best energy per
    # spin within 3 standard errors; their best-energy distributions are also
    # compared by a two-sample Kolmogorov-Smirnov test (p-values reported)
    pm1_same, g_ok, g_n, ks_p = True, 0, 0, []
    for q, a, b in zip(sub, sbest, pbest):
        if jobs[q][2] == "pm1":
            pm1_same &= bool(np.array_equal(a, b))
        else:
            g_n += 1
            se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size) if a.size > 1 else 0.0
            g_ok += int(abs(a.mean() - b.mean()) <= 3 * se + 1e-9 * abs(a.mean()))
            ks_p.append(ks_2samp_p(a, b))
    for i in owned:
        pb.pb_instance_destroy(i)
    return {"workload": "200 instances, seed 7: EA L in {8,12,16,24} / biclique n in {128,...,2048}, +-1 / N(0,1), "
                        "replicas 32..1024 (powers of 2, log-uniform), sweeps log-uniform in [500, 1e4], geometric "
                        "beta 0.1->5.0",
            "updates": upd, "ms": ms, "wall_ms": 1e3 * wall, "value": upd / (ms / 1e3), "unit": UNIT,
            "autotune": {"shapes": len(tuned), "seconds": tune_s},
            "plain_vs_batched_on_every_4th_job": {
                "jobs": len(sub), "updates": sub_upd, "batched_ms": sms, "plain_ms": pms,
                "batched_value": sub_upd / (sms / 1e3), "plain_value": sub_upd / (pms / 1e3), "speedup": pms / sms,
                "pm1_jobs_identical": pm1_same, "gauss_jobs_mean_within_3se": f"{g_ok}/{g_n}",
                "gauss_jobs_ks_2samp": ks_summary(ks_p),
                "plain_forms": "EA plain (one launch per colour and sweep), biclique FP32 CUDA-core"}}


def served_block(pb, stream, n_req: int):
    """Served stream (continuous batching through the request server): Poisson arrivals at
    500 requests/s (seed 11) of jobs drawn like the mixed batch (EA L in {8,12,16,24} /
    biclique n in {128,...,2048}, +-1 / N(0,1), replicas 32..1024) over 48 distinct instances,
    each request with a sweep budget (log-uniform in [50, 1000]) and a target residual energy:
    p E_ref with p = 0.99 (EA) / 0.95 (biclique), E_ref the best energy of a 10^4-sweep,
    256-replica anneal of the instance computed beforehand (10x the largest budget, the stated
    proxy for the ground state); the anneal stops at the target (every replica reached it) or
    at the budget.  Reported: latency from submit to result ready (p50/p99/max), the offered
    load rho = arrival rate / the maximum sustainable rate (completion rate of a burst of
    requests all submitted at once), and the plain per-instance forms on every 20th request
    (one after another, same stop rule): throughput and the residual-energy distributions."""
    import torch
    lam, p_ea, p_bq = 500.0, 0.99, 0.95
    jobs = mixed_jobs(n_req, 11, 50, 1000)
    pool = {}
    for q, j in enumerate(jobs):
        pool.setdefault((j[0], j[1], j[2]), 11000 + len(pool))
    jobs = [(t, sz, law, R, S, pool[(t, sz, law)]) for t, sz, law, R, S, _ in jobs]
    insts, owned = make_instances(pb, jobs, stream)
    key_of = [(j[0], j[1], j[2], j[5]) for j in jobs]
    # E_ref per distinct instance (untimed): one batch of long anneals
    uniq = {}
    for k, inst in zip(key_of, insts):
        uniq.setdefault(k, inst)
    ukeys = list(uniq)
    t0 = time.perf_counter()
    long_s = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, 10000, BETA0, BETA1)
    runs = pb.pb_anneal_batch([uniq[k] for k in ukeys], [long_s] * len(ukeys), [256] * len(ukeys),
                              [77 + q for q in range(len(ukeys))], stream=stream)
    eref = {k: float(pb.pb_energy(r, 256)[1].min()) for k, r in zip(ukeys, runs)}
    for r in runs:
        pb.pb_run_destroy(r)
    eref_s = time.perf_counter() - t0
    scheds = [pb.make_schedule(pb.PB_SCHED_GEOMETRIC, j[4], BETA0, BETA1) for j in jobs]
    target = [(p_ea if j[0] == "ea" else p_bq) * eref[k] for j, k in zip(jobs, key_of)]
    opts = [pb.make_opts(pb.PB_FORM_AUTO, t, pb.PB_FLAG_STOP_AT_TARGET) for t in target]
    seeds = [90000 + q for q in range(n_req)]
    spins = [j[1] ** 3 if j[0] == "ea" else 2 * j[1] for j in jobs]

    def serve(idx, gaps):
        """Submit requests idx at the given inter-arrival gaps (None: all at once); returns
        (span s, per-request best energies, target sweeps, server stats)."""
        torch.cuda.synchronize()
        sv = pb.pb_server_create(max_inflight=512, gather_us=0)
        tickets = [None] * len(idx)
        t_start = time.perf_counter()

        def submitter():
            t = t_start
            for a, q in enumerate(idx):
                if gaps is not None:
                    t += gaps[a]
                    d = t - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                tickets[a] = pb.pb_server_submit(sv, insts[q], scheds[q], jobs[q][3], seeds[q], opts[q])

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        best, hits = {}, {}
        for a, q in enumerate(idx):
            run, _ = pb.pb_server_wait(sv, tickets[a], -1)
            best[q] = pb.pb_energy(run, jobs[q][3])[1]
            hits[q] = pb.pb_target_sweeps(run, jobs[q][3])
            pb.pb_run_destroy(run)
        span = time.perf_counter() - t_start
        st = pb.pb_server_stats_get(sv)
        pb.pb_server_destroy(sv)
        return span, best, hits, st

    allq = list(range(n_req))
    gaps = np.random.default_rng(11).exponential(1.0 / lam, size=n_req)
    span, best, hits, st = serve(allq, gaps)
    # maximum sustainable rate: a burst of the first 4000 requests submitted at once
    burst = allq[: min(4000, n_req)]
    bspan, _, _, bst = serve(burst, None)
    mu_max = len(burst) / bspan
    # plain per-instance forms on every 20th request, one after another
    sub = allq[::20]
    torch.cuda.synchronize()
    pbest = {}
    t0 = time.perf_counter()
    for q in sub:
        f = pb.PB_FORM_PLAIN if jobs[q][0] == "ea" else pb.PB_FORM_CUDACORE
        run = pb.pb_anneal(insts[q], scheds[q], jobs[q][3], seeds[q], pb.make_opts(f, target[q], pb.PB_FLAG_STOP_AT_TARGET),
                           stream=stream)
        pbest[q] = pb.pb_energy(run, jobs[q][3])[1]
        pb.pb_run_destroy(run)
    plain_s = time.perf_counter() - t0
    served_sub_s = sum(1 for _ in sub) / mu_max      # the same requests at the served maximum rate
    pm1_same, g_ok, g_n, ks_p = True, 0, 0, []
    res_served, res_plain = [], []
    for q in sub:
        a, b = best[q], pbest[q]
        e_ref, n_sp = eref[key_of[q]], spins[q]
        res_served.append((a.min() - e_ref) / n_sp)
        res_plain.append((b.min() - e_ref) / n_sp)
        if jobs[q][2] == "pm1":
            pm1_same &= bool(np.array_equal(a, b))
        else:
            g_n += 1
            se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size) if a.size > 1 else 0.0
            g_ok += int(abs(a.mean() - b.mean()) <= 3 * se + 1e-9 * abs(a.mean()))
            ks_p.append(ks_2samp_p(a, b))
    reached = np.array([float((hits[q] >= 0).mean()) for q in allq])
    res_all = np.array([(best[q].min() - eref[key_of[q]]) / spins[q] for q in allq])
    upd = sum(job_updates(j) for j in jobs)
    for i in owned:
        pb.pb_instance_destroy(i)
    return {"workload": "Poisson arrivals 500/s (seed 11) of mixed jobs (EA L in {8,12,16,24} / biclique n in "
                        "{128,...,2048}, +-1 / N(0,1), replicas 32..1024, sweep budgets log-uniform in [50, 1000]), "
                        "48 distinct instances; target p E_ref (p = 0.99 EA, 0.95 biclique), stop at the target",
            "requests": n_req, "seconds": span, "requests_per_s": n_req / span, "offered_req_per_s": lam,
            "budget_updates_per_s": upd / span,
            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms, "max_ms": st.max_ms,
            "rounds": st.rounds, "peak_inflight_bytes": st.peak_inflight_bytes, "failed": st.failed,
            "max_sustainable_req_per_s": mu_max, "offered_load_rho": lam / mu_max,
            "burst": {"requests": len(burst), "seconds": bspan, "p99_ms": bst.p99_ms},
            "e_ref": {"how": "best of a 1e4-sweep geometric 0.1->5.0 anneal with 256 replicas per instance",
                      "instances": len(ukeys), "seconds": eref_s},
            "target": {"requests_all_replicas_reached": int((reached == 1.0).sum()),
                       "mean_fraction_of_replicas_reached": float(reached.mean()),
                       "residual_per_spin_median": float(np.median(res_all)),
                       "residual_per_spin_p90": float(np.quantile(res_all, 0.9))},
            "plain_on_every_20th_request": {
                "requests": len(sub), "plain_seconds": plain_s, "plain_req_per_s": len(sub) / plain_s,
                "served_req_per_s_at_max_rate": mu_max, "speedup": mu_max / (len(sub) / plain_s),
                "served_seconds_equiv": served_sub_s,
                "pm1_requests_identical": pm1_same, "gauss_requests_mean_within_3se": f"{g_ok}/{g_n}",
                "gauss_requests_ks_2samp": ks_summary(ks_p),
                "residual_per_spin_ks_p": ks_2samp_p(np.array(res_served), np.array(res_plain)),
                "residual_per_spin_mean": {"served": float(np.mean(res_served)), "plain": float(np.mean(res_plain))},
                "plain_forms": "EA plain (one launch per colour and sweep), biclique FP32 CUDA-core"}}


# ------------------------------------------------------ next rows (f1-f4)
def extensions_block(pb, stream, peaks):
    """General-graph annealing (odd periodic cube, 3+ colours), parallel tempering on the
    same graph, the sparsified biclique against the dense tensor form at equal sweeps, and
    the Algorithm 1 driver; each timed with CUDA events on the stream it runs on."""
    import torch
    import synth_inputs as syn
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    out = {}
    # f1: odd periodic cube L = 25 (not bipartite), +-J, 1024 replicas, 200 sweeps
    L, R, S = 25, 1024, 200
    eu, ev = syn.graph_periodic_cube(L)
    N = L ** 3
    J = syn.edge_couplings(eu.size, "pm1", 71)
    inst = pb.pb_create_graph_instance(N, eu, ev, J, stream=stream)
    k = pb.pb_instance_colours(inst)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.1, 3.0)
    pb.pb_run_destroy(pb.pb_anneal(inst, pb.make_schedule(pb.PB_SCHED_LINEAR, 2, 0.1, 3.0), R, 1, stream=stream))
    ms, run = timed(lambda: pb.pb_anneal(inst, sc, R, 5, stream=stream))
    kms = pb.pb_run_kernel_ms(run)
    best = float(pb.pb_energy(run, R)[1].min())
    pb.pb_run_destroy(run)
    upd = N * R * S
    deg = 6
    out["csr_k_colour"] = {
        "workload": f"periodic cube L={L} (odd: {k} greedy colours), +-J, {R} replicas, {S} sweeps linear 0.1->3.0",
        "ms": ms, "kernel_ms": kms, "updates_per_s": upd / (kms / 1e3), "best_E_per_spin": best / N,
        "roofline": {"bound": "hbm", "bytes_per_update": deg + 1,
                     "achieved_gbs": upd * (deg + 1) / (kms / 1e3) / 1e9, "peak_gbs": hbm,
                     "frac": upd * (deg + 1) / (kms / 1e3) / 1e9 / hbm, "peak_source": "measured"}}
    # f3: tempering on the same graph: 16 temperatures x 64 chains, 200 sweeps
    M, C = 16, 64
    ladder = np.linspace(0.1, 3.0, M)
    ms, run = timed(lambda: pb.pb_anneal_pt(inst, ladder, S, C, 9, stream=stream))
    kms = pb.pb_run_kernel_ms(run)
    G = M * C
    be = pb.pb_energy(run, G)[1]
    temp, acc = pb.pb_pt_state(run, M, C)
    pb.pb_run_destroy(run)
    out["parallel_tempering"] = {
        "workload": f"same cube, ladder linear 0.1..3.0 with {M} rungs, {C} chains, {S} sweeps",
        "ms": ms, "kernel_ms": kms, "updates_per_s": N * G * S / (kms / 1e3), "best_E_per_spin": float(be.min()) / N,
        "exchange_acceptance": [float(a) / (C * (S // 2)) for a in acc]}
    pb.pb_instance_destroy(inst)
    # f4: sparsified biclique n = 512 on the general-graph path vs the dense tensor form, at several
    # copy strengths (the copies of a vertex must agree for the projection to keep the energy)
    n, R, S = 512, 256, 300
    Jb = pb.pb_generate_biclique(n, pb.PB_DIST_PM1, 72)
    dinst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, Jb, None, n=n, stream=stream)
    sc = pb.make_schedule(pb.PB_SCHED_LINEAR, S, 0.35, 3.5)
    ms_d, run = timed(lambda: pb.pb_anneal(dinst, sc, R, 3, stream=stream))
    dense_best = float(pb.pb_energy(run, R)[1].min())
    pb.pb_run_destroy(run)
    by_strength = []
    for cs in (2, 6, 16):
        sp = pb.pb_sparsify_biclique(Jb, 4, cs)
        sinst = pb.pb_create_graph_instance(sp["N"], sp["eu"], sp["ev"], sp["J"], None, sp["colour"], stream=stream)
        ms_s, run = timed(lambda: pb.pb_anneal(sinst, sc, R, 3, stream=stream))
        bst = pb.pb_best_states(run, R, sp["N"])
        pb.pb_run_destroy(run)
        pb.pb_instance_destroy(sinst)
        proj = pb.pb_sparse_project(sp["copy_of"], 2 * n, bst)
        F = pb.pb_fields(dinst, proj, stream=stream)  # biclique energies of the projected states: -(sum m F)/2
        e_proj = -0.5 * (proj.astype(np.float64) * F.astype(np.float64)).sum(axis=1)
        # copy agreement: fraction of copies whose spin equals their vertex's projected (majority) spin
        agree = float((bst == proj[:, sp["copy_of"]]).mean())
        by_strength.append({"copy_strength": cs, "spins": sp["N"], "sparse_ms": ms_s,
                            "best_E_per_spin_projected": float(e_proj.min()) / (2 * n),
                            "copy_agreement": agree})
    pb.pb_instance_destroy(dinst)
    out["sparsified_biclique"] = {
        "workload": f"biclique n={n} +-J, copy graph (<= 4 edges per copy, copy edges of strength c), "
                    f"{R} replicas, {S} sweeps linear 0.35->3.5; projection by majority of copies",
        "dense_tensor_ms": ms_d, "best_E_per_spin_dense": dense_best / (2 * n), "by_copy_strength": by_strength}
    # f2: Algorithm 1 on an EA L = 8 +-J cube
    J8 = pb.pb_generate_ea(8, pb.PB_DIST_PM1, 73)
    einst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J8, None, L=8, stream=stream)
    run = pb.pb_anneal(einst, pb.make_schedule(pb.PB_SCHED_LINEAR, 2000, 0.35, 3.5), 256, 4, stream=stream)
    G0 = float(pb.pb_energy(run, 256)[1].min())
    pb.pb_run_destroy(run)
    t0 = time.perf_counter()
    r = pb.pb_find_imin(einst, G0, 0.97, 0.9, i_start=10, i_step=20, trials=128, i_max=4000, budgets_per_launch=8,
                        seed=77, stream=stream)
    dt = time.perf_counter() - t0
    pb.pb_instance_destroy(einst)
    out["algorithm1"] = {"workload": "EA L=8 +-J, G = best of 256 replicas x 2000 sweeps, p = 0.97, p_succ = 0.9, "
                                     "128 trials, budgets 10, 30, ... (8 per launch)",
                         "i_min": r.i_min, "fails": r.fails, "budgets_tried": r.budgets_tried,
                         "launches": r.launches, "seconds": dt}
    return out


# ------------------------------------------------- small profiling cases
CASES = {
    # name: (topology, L or n, law, replicas, sweeps, form)
    "ea-L32-pm1-small": ("ea", 32, "pm1", 608, 50, "resident"),
    "ea-L32-gauss-small": ("ea", 32, "gauss", 608, 50, "resident"),
    "ea-L16-pm1-small": ("ea", 16, "pm1", 2432, 50, "resident"),
    "ea-L16-gauss-small": ("ea", 16, "gauss", 2432, 50, "resident"),
    "ea-L24-pm1-small": ("ea", 24, "pm1", 608, 50, "resident"),      # generic tile (WT = 1)
    "ea-L12-pm1-small": ("ea", 12, "pm1", 2432, 50, "resident"),     # generic tile (WT = 4)
    "ea-L24-gauss-small": ("ea", 24, "gauss", 608, 50, "resident"),  # generic tile, FP32
    "bq-n4096-R4096-pm1-tensor": ("bq", 4096, "pm1", 4096, 2, "tensor"),
    "bq-n4096-R4096-gauss-tensor": ("bq", 4096, "gauss", 4096, 2, "tensor"),
    "bq-n4096-R1024-pm1-cudacore": ("bq", 4096, "pm1", 1024, 1, "cudacore"),
    "bq-n1024-R1024-pm1-tensor": ("bq", 1024, "pm1", 1024, 4, "tensor"),
    "bq-n4096-R4096-pm1-tensor-s200": ("bq", 4096, "pm1", 4096, 200, "tensor"),
    "bq-n4096-R4096-gauss-tensor-s100": ("bq", 4096, "gauss", 4096, 100, "tensor"),
    "csr-cube25-R1024-pm1": ("csr", 25, "pm1", 1024, 50, "plain"),
}


def run_case(name, sweeps=None):
    """One launch of the hot-path kernel on a small case (152 tiles: one wave), for ncu;
    `sweeps` overrides the case's sweep count."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_23419_gb300 import native as pb
    topo, size, law, R, S, form = CASES[name]
    if sweeps:
        S = sweeps
    dist = {"pm1": pb.PB_DIST_PM1, "gauss": pb.PB_DIST_GAUSS, "unif": pb.PB_DIST_UNIF}[law]
    forms = {"resident": pb.PB_FORM_RESIDENT, "plain": pb.PB_FORM_PLAIN, "cudacore": pb.PB_FORM_CUDACORE,
             "tensor": pb.PB_FORM_TENSOR}
    if topo == "ea":
        J = pb.pb_generate_ea(size, dist, 3)
        inst = pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=size)
    elif topo == "csr":
        import synth_inputs as syn
        eu, ev = syn.graph_periodic_cube(size)
        inst = pb.pb_create_graph_instance(size ** 3, eu, ev, syn.edge_couplings(eu.size, law, 3))
    else:
        J = pb.pb_generate_biclique(size, dist, 3)
        inst = pb.pb_create_instance(pb.PB_TOPO_BICLIQUE, J, None, n=size)
    sc = pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S, 0.1, 5.0)
    run = pb.pb_anneal(inst, sc, R, 7, pb.make_opts(forms[form]))
    ms = pb.pb_run_kernel_ms(run)
    dev_ms = pb.pb_run_device_ms(run)
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "kernel_ms": ms, "device_ms": dev_ms}))
    pb.pb_run_destroy(run)
    pb.pb_instance_destroy(inst)


# --------------------------------------------------------------- ours
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-biclique", action="store_true", help="skip the biclique tensor-core measurement")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 200-instance mixed batch")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip general graphs, tempering, sparsified biclique and Algorithm 1")
    ap.add_argument("--no-serve", action="store_true", help="skip the served Poisson stream")
    ap.add_argument("--serve-requests", type=int, default=15000, help="requests of the served stream")
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="run one small launch of a hot-path kernel (for ncu) and exit")
    ap.add_argument("--case-sweeps", type=int, default=None, help="sweeps of the --case run")
    args = ap.parse_args()
    if args.case:
        run_case(args.case, args.case_sweeps)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_23419_gb300 import native as pb

    stream = torch.cuda.Stream()   # a non-default stream: the batch launch is captured into a CUDA graph
    torch.cuda.set_stream(stream)
    Js = [pb.pb_generate_ea(L, pb.PB_DIST_PM1 if law == "pm1" else pb.PB_DIST_GAUSS, seed) for L, law, seed in JOBS]
    insts = [pb.pb_create_instance(pb.PB_TOPO_EA3D, J, None, L=L, stream=stream) for J, (L, _, _) in zip(Js, JOBS)]
    scheds = [pb.make_schedule(pb.PB_SCHED_GEOMETRIC, S_SWEEPS, BETA0, BETA1) for _ in JOBS]
    seeds = rank_seeds(rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(opts=None):
        runs = pb.pb_anneal_batch(insts, scheds, [R_REPLICAS] * len(JOBS), seeds, opts, stream=stream)
        return runs

    # warm-up; the best energies found give the time-to-target reference E_ref
    eref = [math.inf] * len(JOBS)
    for _ in range(args.warmup):
        runs = one_step()
        for q, r in enumerate(runs):
            _, be, _ = pb.pb_energy(r, R_REPLICAS)
            eref[q] = min(eref[q], float(be.min()))
            pb.pb_run_destroy(r)
    p_target = 0.99
    opts = [pb.make_opts(pb.PB_FORM_RESIDENT, p_target * e) for e in eref]

    # ---- timed region: device-resident inputs ----
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms, kern_ms, hit = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        runs = one_step(opts)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(pb.pb_run_kernel_ms(runs[0]))
        hit.append([pb.pb_target_sweeps(r, R_REPLICAS) for r in runs])
        for r in runs:
            pb.pb_run_destroy(r)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_max_ms, upd = aggregate_ranks(sum(step_ms), updates_per_step() * args.steps, dist, device="cuda")
    value = upd / (t_max_ms / 1e3)
    ms_per_step = t_max_ms / args.steps

    # ---- end to end through the C ABI with host buffers ----
    pinned = [torch.from_numpy(J).pin_memory() for J in Js]
    h2d = sum(J.nbytes for J in Js)
    d2h = 0
    e2e_ms = []
    for _ in range(max(1, min(3, args.steps))):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ins = [pb.pb_create_instance(pb.PB_TOPO_EA3D, P.numpy(), None, L=L, stream=stream)
               for P, (L, _, _) in zip(pinned, JOBS)]
        runs = pb.pb_anneal_batch(ins, scheds, [R_REPLICAS] * len(JOBS), seeds, stream=stream)
        d2h = 0
        for r, (L, _, _) in zip(runs, JOBS):
            fe, be, bs = pb.pb_energy(r, R_REPLICAS)
            st = pb.pb_best_states(r, R_REPLICAS, L ** 3)
            d2h += fe.nbytes + be.nbytes + bs.nbytes + st.nbytes
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        for r in runs:
            pb.pb_run_destroy(r)
        for i in ins:
            pb.pb_instance_destroy(i)
    e2e_value = updates_per_step() * world / (statistics.median(e2e_ms) / 1e3)

    # ---- roofline of the dominant kernels (the persistent resident kernels of the step) ----
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    k_ms = statistics.mean(kern_ms)
    achieved = updates_per_step() / (k_ms / 1e3) / 1e9          # Gupdate/s per launch
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # measured ALU ceiling: a kernel that draws exactly the tiles' random words (one
    # Philox4x32-10 word per update, same counters) and nothing else
    ceil_gups = philox_ceiling(pb, stream) / 1e9
    # derived IMAD bound, for context: 20 32x32->64 multiplies per 4 updates, the high
    # and low halves as two IMAD issues at 64 IMAD/clk/SM -> 6.4 updates/clk/SM
    imad_peak = n_sm * 64.0 / 10.0 * sm_max * 1e6 / 1e9           # Gupdate/s
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    traffic = profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": ceil_gups, "unit": "Gupdate/s",
                "frac": achieved / ceil_gups, "traffic": traffic,
                "traffic_source": "profiles/ea_resident_batch_dram.md (ncu dram__bytes_read+write, both kernels of one step)",
                "peak_source": "measured: Philox-only ceiling kernel (pb_philox_ceiling: the tiles' decision words, "
                               "one per update, nothing else), best of 3, this run",
                "kernel": "ea_resident_kernel<f32> then ea_resident_kernel<+-1> (chained; events around both)",
                "kernel_ms": k_ms,
                "imad_bound": {"peak": imad_peak, "frac": achieved / imad_peak, "sms": n_sm,
                               "source": f"derived: {n_sm} SMs (device query) x 64 IMAD/clk x max SM clock / "
                                         "10 IMAD per update"},
                "hbm_equiv": {"bytes_per_update": 2, "achieved_gbs": achieved * 2, "peak_gbs": hbm,
                              "frac": achieved * 2 / hbm, "peak_source": "measured (peak file)"}}
    dense = measure_dense_peaks()
    peaks = dict(peaks)
    peaks["fp8_tflops_measured"] = dense.get("fp8_tflops")
    line_peaks = {"fp8_tflops": dense.get("fp8_tflops"), "bf16_tflops_this_run": dense.get("bf16_tflops"),
                  "bf16_tflops_peak_file": peaks.get("bf16_tflops"), "how": dense.get("fp8_how", dense.get("fp8_error")),
                  "n": dense["n"], "reps": dense["reps"]}

    # ---- time to target (p = 0.99 of the best warm-up energy, 90% of replicas) ----
    ttt = []
    for q, (L, law, _) in enumerate(JOBS):
        hs = np.array(hit[-1][q])
        ok = np.sort(hs[hs >= 0])
        need = int(math.ceil(0.9 * R_REPLICAS))
        s90 = int(ok[need - 1]) if ok.size >= need else None
        ttt.append({"job": f"L{L}-{law}", "E_ref": eref[q], "target": p_target * eref[q],
                    "sweeps_to_90pct": s90,
                    "ms_estimate": None if s90 is None else ms_per_step * (s90 + 1) / S_SWEEPS})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/int32 (+-1), f32 (Gaussian)", "data": "synthetic", "config": CONFIG,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (len({j[1] for j in JOBS}) + 4 * len(JOBS)),
            "roofline": roofline, "time_to_target": ttt, "measured_peaks": line_peaks}

    # ---- plain per-instance form on the same inputs (one pass) ----
    if not args.no_plain and rank == 0:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        runs = [pb.pb_anneal(i, s, R_REPLICAS, sd, pb.make_opts(pb.PB_FORM_PLAIN), stream=stream)
                for i, s, sd in zip(insts, scheds, seeds)]
        e1.record(stream)
        e1.synchronize()
        pms = e0.elapsed_time(e1)
        for r in runs:
            pb.pb_run_destroy(r)
        pv = updates_per_step() / (pms / 1e3)
        line["plain_form"] = {"value": pv, "unit": UNIT, "ms_per_step": pms, "speedup_of_batched": value / world / pv}

    if rank == 0:
        line["config1"] = config1_block(pb, stream)
    if rank == 0 and not args.no_biclique:
        line["biclique"] = biclique_block(pb, stream, peaks)
        line["biclique_sweep"] = biclique_sweep_block(pb, stream, peaks)
    if rank == 0 and not args.no_extensions:
        line["next_rows"] = extensions_block(pb, stream, peaks)
    if rank == 0 and not args.no_mixed:
        line["mixed_batch"] = mixed_block(pb, stream)
    if rank == 0 and not args.no_serve:
        line["served"] = served_block(pb, stream, args.serve_requests)

    if rank == 0 and not args.no_cpu and world == 1:
        from oracle import oracle as orc
        orc.build()
        u, dt = oracle_sample(3000)
        line["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "replica 0 of each of the 4 jobs, first 3000 sweeps of the schedule"}
        cores = max(1, os.cpu_count() or 1)
        ua, wa = oracle_sample_all_cores(3000, cores)
        line["cpu_baseline"]["all_cores"] = {
            "value": ua / wa, "unit": UNIT, "cores": cores, "kind": "oracle, one process per core",
            "sample": f"replicas 0..{cores - 1} (one per process) of each of the 4 jobs, first 3000 sweeps"}
        uc, tc = oracle_config1()
        line["cpu_baseline"]["config1"] = {
            "value": uc / tc, "unit": UNIT, "seconds": tc, "cores": 1, "kind": "oracle",
            "sample": "the whole small-cube run (EA L = 6, 64 replicas, 1000 sweeps), as config1 times it on the GPU"}
    for i in insts:
        pb.pb_instance_destroy(i)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Thin ctypes binding of the C ABI in ``include/pbit.h`` (libpbit.so).

Argument marshalling only: every step of the annealing path runs in the CUDA
library.  Function names follow the C ABI.  Arrays are numpy arrays on the
host; CUDA streams come from PyTorch (``torch.cuda.current_stream()``) or as
raw ``cudaStream_t`` integers.  There is no CPU fallback: if the library is
missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _build

PB_OK, PB_EINVAL, PB_ECOLOUR, PB_ENOMEM, PB_EDEVICE, PB_ETIMEOUT, PB_EBUSY, PB_EUNSUPPORTED = range(8)
PB_TOPO_EA3D, PB_TOPO_BICLIQUE, PB_TOPO_CSR = 0, 1, 2
PB_J_PM1_I8, PB_J_F32 = 0, 1
PB_DIST_PM1, PB_DIST_GAUSS, PB_DIST_UNIF = 0, 1, 2
PB_SCHED_LINEAR, PB_SCHED_GEOMETRIC, PB_SCHED_EXPLICIT = 0, 1, 2
PB_FORM_AUTO, PB_FORM_PLAIN, PB_FORM_RESIDENT, PB_FORM_CUDACORE, PB_FORM_TENSOR = range(5)
PB_FLAG_TEST_EXPIRE_WAITS = 0x40000000  # failure-path test hook (see include/pbit.h)
PB_FLAG_STOP_AT_TARGET = 0x1  # freeze each replica's best at the target, end the run once all reached it
PB_NOALLOC_BAD_COUPLINGS = -2  # best_sweep of pb_anneal_ea_noalloc when J_dev holds a value other than +-1

_ERRNAMES = {0: "PB_OK", 1: "PB_EINVAL", 2: "PB_ECOLOUR", 3: "PB_ENOMEM", 4: "PB_EDEVICE", 5: "PB_ETIMEOUT",
             6: "PB_EBUSY", 7: "PB_EUNSUPPORTED"}


class PbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(status, status)}: {msg}")
        self.status = status


class pb_instance_desc(ctypes.Structure):
    _fields_ = [("topo", ctypes.c_int32), ("L", ctypes.c_int32), ("n", ctypes.c_int32), ("jtype", ctypes.c_int32),
                ("J", ctypes.c_void_p), ("h", ctypes.c_void_p), ("colour", ctypes.c_void_p)]


class pb_graph_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("jtype", ctypes.c_int32), ("n_edges", ctypes.c_int64), ("eu", ctypes.c_void_p),
                ("ev", ctypes.c_void_p), ("J", ctypes.c_void_p), ("h", ctypes.c_void_p), ("colour", ctypes.c_void_p)]


class pb_imin_opts(ctypes.Structure):
    _fields_ = [("ground", ctypes.c_double), ("p", ctypes.c_double), ("p_succ", ctypes.c_double),
                ("i_start", ctypes.c_int32), ("i_step", ctypes.c_int32), ("i_max", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("beta_i", ctypes.c_double), ("beta_f", ctypes.c_double),
                ("budgets_per_launch", ctypes.c_int32), ("form", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class pb_imin_result(ctypes.Structure):
    _fields_ = [("i_min", ctypes.c_int32), ("fails", ctypes.c_int32), ("budgets_tried", ctypes.c_int32),
                ("launches", ctypes.c_int32)]


class pb_schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_sweeps", ctypes.c_int32), ("step_duration", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
                ("betas", ctypes.c_void_p)]


class pb_anneal_opts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("flags", ctypes.c_int32), ("target_energy", ctypes.c_double)]


class pb_tune_result(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("tile_width", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("candidate_form", ctypes.c_int32 * 8), ("candidate_wt", ctypes.c_int32 * 8),
                ("probe_ms", ctypes.c_float * 8)]


class pb_server_opts(ctypes.Structure):
    _fields_ = [("max_device_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32), ("gather_us", ctypes.c_int32)]


class pb_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("inflight", ctypes.c_int64),
                ("inflight_bytes", ctypes.c_int64), ("peak_inflight_bytes", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libpbit.so; raise if it has not been built (``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "pb_version": ([], ctypes.c_char_p),
        "pb_status_string": ([st], ctypes.c_char_p),
        "pb_last_error": ([], ctypes.c_char_p),
        "pb_generate_ea": ([I32, I32, U64, P, I64], st),
        "pb_generate_biclique": ([I32, I32, U64, P, I64], st),
        "pb_create_instance": ([P, P, P], st),
        "pb_instance_destroy": ([P], None),
        "pb_instance_spins": ([P], I64),
        "pb_anneal": ([P, P, I32, U64, P, P], st),
        "pb_anneal_ex": ([P, P, I32, U64, P, P, P], st),
        "pb_anneal_batch": ([I32, P, P, P, P, P, P, P], st),
        "pb_wait": ([P, I32], st),
        "pb_query": ([P], st),
        "pb_energy": ([P, P, P, P], st),
        "pb_best_states": ([P, P, I64], st),
        "pb_final_states": ([P, P, I64], st),
        "pb_target_sweeps": ([P, P], st),
        "pb_run_device_ms": ([P, P], st),
        "pb_run_kernel_ms": ([P, P], st),
        "pb_run_destroy": ([P], None),
        "pb_fields": ([P, P, I32, P, I64, P], st),
        "pb_fields_ex": ([P, P, I32, I32, P, I64, P], st),
        "pb_anneal_ea_noalloc": ([I32, P, P, I32, U64, P, P, P, P, P, P], st),
        "pb_philox_ceiling": ([I32, I32, P, P, P], st),
        "pb_create_graph_instance": ([P, P, P], st),
        "pb_greedy_colouring": ([I32, I64, P, P, P], I32),
        "pb_instance_colours": ([P], I32),
        "pb_find_imin": ([P, P, P, P], st),
        "pb_anneal_pt": ([P, P, I32, I32, I32, U64, P, P], st),
        "pb_anneal_resume": ([P, P, I32, U64, I32, P, P, P, P, P, P], st),
        "pb_pt_state": ([P, P, P], st),
        "pb_sparsify_biclique": ([I32, I32, P, I32, I32, P, P, P, P, P, P, I64, I32], I64),
        "pb_sparse_project": ([I32, P, I32, I32, P, P], I32),
        "pb_autotune": ([P, I32, I32, P, P], st),
        "pb_autotune_clear": ([], None),
        "pb_run_footprint": ([P, P, I32, P], I64),
        "pb_server_create": ([P, P], st),
        "pb_server_submit": ([P, P, P, I32, U64, P, P], st),
        "pb_server_wait": ([P, I64, I32, P, P], st),
        "pb_server_stats_get": ([P, P], st),
        "pb_server_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != PB_OK:
        raise PbError(status, load().pb_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ basics
def pb_version() -> str:
    return load().pb_version().decode()


def pb_status_string(status: int) -> str:
    return load().pb_status_string(status).decode()


def pb_last_error() -> str:
    return load().pb_last_error().decode()


def pb_generate_ea(L: int, dist: int, seed: int) -> np.ndarray:
    """Seeded EA couplings [3, L^3]: int8 for PB_DIST_PM1, float32 otherwise."""
    J = np.empty((3, L ** 3), dtype=np.int8 if dist == PB_DIST_PM1 else np.float32)
    _check(load().pb_generate_ea(L, dist, seed, _ptr(J), J.nbytes))
    return J


def pb_generate_biclique(n: int, dist: int, seed: int) -> np.ndarray:
    J = np.empty((n, n), dtype=np.int8 if dist == PB_DIST_PM1 else np.float32)
    _check(load().pb_generate_biclique(n, dist, seed, _ptr(J), J.nbytes))
    return J


# --------------------------------------------------------------- instances
def pb_create_instance(topo: int, J: np.ndarray, h: np.ndarray | None = None, colour: np.ndarray | None = None,
                       L: int = 0, n: int = 0, stream=None) -> ctypes.c_void_p:
    pm1 = J.dtype == np.int8
    J = np.ascontiguousarray(J)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int8 if pm1 else np.float32)
    cc = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    d = pb_instance_desc(topo=topo, L=L, n=n, jtype=PB_J_PM1_I8 if pm1 else PB_J_F32, J=_ptr(J), h=_ptr(hh),
                         colour=_ptr(cc))
    out = ctypes.c_void_p()
    _check(load().pb_create_instance(ctypes.byref(d), _stream(stream), ctypes.byref(out)))
    return out


def pb_create_graph_instance(N: int, eu: np.ndarray, ev: np.ndarray, J: np.ndarray, h: np.ndarray | None = None,
                             colour: np.ndarray | None = None, stream=None) -> ctypes.c_void_p:
    """General sparse instance: edges (eu[e], ev[e]) with couplings J[e] (int8 +-1 or float32)."""
    pm1 = J.dtype == np.int8
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    J = np.ascontiguousarray(J)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.int8 if pm1 else np.float32)
    cc = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    d = pb_graph_desc(N=N, jtype=PB_J_PM1_I8 if pm1 else PB_J_F32, n_edges=eu.size, eu=_ptr(eu), ev=_ptr(ev),
                      J=_ptr(J), h=_ptr(hh), colour=_ptr(cc))
    out = ctypes.c_void_p()
    _check(load().pb_create_graph_instance(ctypes.byref(d), _stream(stream), ctypes.byref(out)))
    return out


def pb_greedy_colouring(N: int, eu: np.ndarray, ev: np.ndarray):
    """(colour[N], number of colours); host only."""
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    col = np.empty(N, np.int32)
    k = int(load().pb_greedy_colouring(N, eu.size, _ptr(eu), _ptr(ev), _ptr(col)))
    if k < 0:
        raise PbError(PB_EINVAL, "invalid graph")
    return col, k


def pb_instance_colours(inst) -> int:
    return int(load().pb_instance_colours(inst))


def pb_instance_destroy(inst):
    if inst:
        load().pb_instance_destroy(inst)


def pb_instance_spins(inst) -> int:
    return int(load().pb_instance_spins(inst))


def make_schedule(kind: int, n_sweeps: int, beta0: float = 0.0, beta1: float = 0.0, step_duration: int = 1,
                  betas: np.ndarray | None = None):
    """pb_schedule (the explicit betas array is kept alive on the returned object)."""
    b = None if betas is None else np.ascontiguousarray(betas, dtype=np.float64)
    s = pb_schedule(kind=kind, n_sweeps=n_sweeps, step_duration=step_duration, reserved=0, beta0=beta0,
                    beta1=beta1, betas=_ptr(b))
    s._keep = b
    return s


def make_opts(form: int = PB_FORM_AUTO, target_energy: float = math.nan, flags: int = 0):
    return pb_anneal_opts(form=form, flags=flags, target_energy=target_energy)


# ------------------------------------------------------------------- runs
def pb_anneal(inst, sched: pb_schedule, replicas: int, seed: int, opts: pb_anneal_opts | None = None,
              stream=None) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    lib = load()
    if opts is None:
        _check(lib.pb_anneal(inst, ctypes.byref(sched), replicas, seed, _stream(stream), ctypes.byref(out)))
    else:
        _check(lib.pb_anneal_ex(inst, ctypes.byref(sched), replicas, seed, ctypes.byref(opts), _stream(stream),
                                ctypes.byref(out)))
    return out


def pb_anneal_ex(inst, sched: pb_schedule, replicas: int, seed: int, opts: pb_anneal_opts,
                 stream=None) -> ctypes.c_void_p:
    return pb_anneal(inst, sched, replicas, seed, opts, stream)


def pb_anneal_batch(insts, scheds, replicas, seeds, opts=None, stream=None):
    k = len(insts)
    ia = (ctypes.c_void_p * k)(*[i.value for i in insts])
    sa = (pb_schedule * k)(*scheds)
    ra = (ctypes.c_int32 * k)(*replicas)
    ea = (ctypes.c_uint64 * k)(*seeds)
    oa = None if opts is None else (pb_anneal_opts * k)(*opts)
    outs = (ctypes.c_void_p * k)()
    _check(load().pb_anneal_batch(k, ia, sa, ra, ea, oa, _stream(stream), outs))
    return [ctypes.c_void_p(o) for o in outs]


def pb_wait(run, timeout_ms: int = -1) -> int:
    return int(load().pb_wait(run, timeout_ms))


def pb_query(run) -> int:
    return int(load().pb_query(run))


def pb_energy(run, replicas: int):
    fe = np.empty(replicas, np.float64)
    be = np.empty(replicas, np.float64)
    bs = np.empty(replicas, np.int32)
    _check(load().pb_energy(run, _ptr(fe), _ptr(be), _ptr(bs)))
    return fe, be, bs


def pb_best_states(run, replicas: int, N: int) -> np.ndarray:
    out = np.empty((replicas, N), np.int8)
    _check(load().pb_best_states(run, _ptr(out), out.nbytes))
    return out


def pb_final_states(run, replicas: int, N: int) -> np.ndarray:
    out = np.empty((replicas, N), np.int8)
    _check(load().pb_final_states(run, _ptr(out), out.nbytes))
    return out


def pb_target_sweeps(run, replicas: int) -> np.ndarray:
    out = np.empty(replicas, np.int32)
    _check(load().pb_target_sweeps(run, _ptr(out)))
    return out


def pb_run_device_ms(run) -> float:
    ms = ctypes.c_float()
    _check(load().pb_run_device_ms(run, ctypes.byref(ms)))
    return float(ms.value)


def pb_run_kernel_ms(run) -> float:
    ms = ctypes.c_float()
    _check(load().pb_run_kernel_ms(run, ctypes.byref(ms)))
    return float(ms.value)


def pb_run_destroy(run):
    if run:
        load().pb_run_destroy(run)


def pb_fields(inst, states: np.ndarray, stream=None) -> np.ndarray:
    return pb_fields_ex(inst, states, PB_FORM_AUTO, stream)


def pb_fields_ex(inst, states: np.ndarray, form: int, stream=None) -> np.ndarray:
    states = np.ascontiguousarray(states, dtype=np.int8)
    R, N = states.shape
    out = np.empty((R, N), np.float32)
    _check(load().pb_fields_ex(inst, _ptr(states), R, form, _ptr(out), out.nbytes, _stream(stream)))
    return out


def pb_anneal_ea_noalloc(L: int, J_dev: int, sched: pb_schedule, replicas: int, seed: int, best_E_dev: int,
                         best_sweep_dev: int, best_states_dev: int, final_E_dev: int, final_states_dev: int,
                         stream=None):
    """EA +-1 anneal into caller-owned device buffers (raw device pointers); allocates nothing."""
    _check(load().pb_anneal_ea_noalloc(L, ctypes.c_void_p(J_dev), ctypes.byref(sched), replicas, seed,
                                       ctypes.c_void_p(best_E_dev), ctypes.c_void_p(best_sweep_dev),
                                       ctypes.c_void_p(best_states_dev), ctypes.c_void_p(final_E_dev),
                                       ctypes.c_void_p(final_states_dev), _stream(stream)))


def pb_philox_ceiling(sweeps: int, blocks: int = 0, stream=None):
    """(kernel ms, p-bit updates whose random words it drew) of the random-word ceiling kernel."""
    ms = ctypes.c_float()
    upd = ctypes.c_double()
    _check(load().pb_philox_ceiling(sweeps, blocks, _stream(stream), ctypes.byref(ms), ctypes.byref(upd)))
    return float(ms.value), float(upd.value)


# ------------------------------------------------------- parallel tempering
def pb_anneal_pt(inst, ladder, n_sweeps: int, chains: int, seed: int, stream=None) -> ctypes.c_void_p:
    lad = np.ascontiguousarray(ladder, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(load().pb_anneal_pt(inst, _ptr(lad), lad.size, n_sweeps, chains, seed, _stream(stream), ctypes.byref(out)))
    return out


def pb_anneal_resume(inst, sched: pb_schedule, replicas: int, seed: int, first_sweep: int, state: np.ndarray,
                     best_state: np.ndarray, best_E: np.ndarray, best_sweep: np.ndarray, stream=None) -> ctypes.c_void_p:
    """Continue an anneal of a general sparse instance at sweep `first_sweep` from the
    given state and running best (host arrays, copied before the call returns)."""
    st = np.ascontiguousarray(state, dtype=np.int8)
    bst = np.ascontiguousarray(best_state, dtype=np.int8)
    be = np.ascontiguousarray(best_E, dtype=np.float64)
    bs = np.ascontiguousarray(best_sweep, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(load().pb_anneal_resume(inst, ctypes.byref(sched), replicas, seed, first_sweep, _ptr(st), _ptr(bst), _ptr(be),
                                   _ptr(bs), _stream(stream), ctypes.byref(out)))
    return out


def pb_pt_state(run, M: int, chains: int):
    """(final temperature index of every slot [M * chains], accepted exchanges per pair [M - 1])."""
    t = np.empty(M * chains, np.int32)
    a = np.zeros(max(M - 1, 1), np.int64)
    _check(load().pb_pt_state(run, _ptr(t), _ptr(a)))
    return t, a[: M - 1]


# ------------------------------------------------------- sparsified biclique
def pb_sparsify_biclique(J: np.ndarray, per_copy: int = 4, copy_strength: int = 2):
    """Copy graph of the biclique with couplings J [n][n] (int8 or float32):
    dict(N, eu, ev, J, colour, copy_of)."""
    J = np.ascontiguousarray(J)
    n = J.shape[0]
    jt = PB_J_PM1_I8 if J.dtype == np.int8 else PB_J_F32
    N = ctypes.c_int32()
    lib = load()
    E = int(lib.pb_sparsify_biclique(n, jt, _ptr(J), per_copy, copy_strength, ctypes.byref(N), None, None, None, None,
                                     None, 0, 0))
    if E < 0:
        raise PbError(PB_EINVAL, "invalid sparsification arguments")
    eu = np.empty(E, np.int32)
    ev = np.empty(E, np.int32)
    Jo = np.empty(E, np.int8 if jt == PB_J_PM1_I8 else np.float32)
    col = np.empty(N.value, np.int32)
    cof = np.empty(N.value, np.int32)
    got = int(lib.pb_sparsify_biclique(n, jt, _ptr(J), per_copy, copy_strength, ctypes.byref(N), _ptr(eu), _ptr(ev),
                                       _ptr(Jo), _ptr(col), _ptr(cof), E, N.value))
    if got != E:
        raise PbError(PB_EINVAL, "sparsification failed")
    return dict(N=N.value, eu=eu, ev=ev, J=Jo, colour=col, copy_of=cof)


def pb_sparse_project(copy_of: np.ndarray, n_orig: int, states: np.ndarray) -> np.ndarray:
    states = np.ascontiguousarray(states, dtype=np.int8)
    R, Ns = states.shape
    out = np.empty((R, n_orig), np.int8)
    cof = np.ascontiguousarray(copy_of, dtype=np.int32)
    if load().pb_sparse_project(Ns, _ptr(cof), n_orig, R, _ptr(states), _ptr(out)) != 0:
        raise PbError(PB_EINVAL, "invalid projection arguments")
    return out


# ------------------------------------------------------- Algorithm 1 driver
def pb_find_imin(inst, ground: float, p: float, p_succ: float, i_start: int, i_step: int, trials: int,
                 beta_i: float = 0.35, beta_f: float = 3.5, i_max: int = 0, budgets_per_launch: int = 0,
                 form: int = PB_FORM_AUTO, seed: int = 0, stream=None) -> pb_imin_result:
    o = pb_imin_opts(ground=ground, p=p, p_succ=p_succ, i_start=i_start, i_step=i_step, i_max=i_max, trials=trials,
                     beta_i=beta_i, beta_f=beta_f, budgets_per_launch=budgets_per_launch, form=form, seed=seed)
    r = pb_imin_result()
    _check(load().pb_find_imin(inst, ctypes.byref(o), _stream(stream), ctypes.byref(r)))
    return r


# ------------------------------------------------------- autotuner, server
def pb_autotune(inst, replicas: int, probe_sweeps: int = 8, stream=None) -> pb_tune_result:
    r = pb_tune_result()
    _check(load().pb_autotune(inst, replicas, probe_sweeps, _stream(stream), ctypes.byref(r)))
    return r


def pb_autotune_clear():
    load().pb_autotune_clear()


def pb_run_footprint(inst, sched: pb_schedule, replicas: int, opts: pb_anneal_opts | None = None) -> int:
    return int(load().pb_run_footprint(inst, ctypes.byref(sched), replicas,
                                       None if opts is None else ctypes.byref(opts)))


def pb_server_create(max_device_bytes: int = 0, max_inflight: int = 0, gather_us: int = 0) -> ctypes.c_void_p:
    o = pb_server_opts(max_device_bytes=max_device_bytes, max_inflight=max_inflight, gather_us=gather_us)
    out = ctypes.c_void_p()
    _check(load().pb_server_create(ctypes.byref(o), ctypes.byref(out)))
    return out


def pb_server_submit(sv, inst, sched: pb_schedule, replicas: int, seed: int,
                     opts: pb_anneal_opts | None = None) -> int:
    t = ctypes.c_int64()
    _check(load().pb_server_submit(sv, inst, ctypes.byref(sched), replicas, seed,
                                   None if opts is None else ctypes.byref(opts), ctypes.byref(t)))
    return int(t.value)


def pb_server_wait(sv, ticket: int, timeout_ms: int = -1):
    """(run, latency_ms) of a finished ticket; the caller owns the run."""
    run = ctypes.c_void_p()
    lat = ctypes.c_double()
    _check(load().pb_server_wait(sv, ticket, timeout_ms, ctypes.byref(run), ctypes.byref(lat)))
    return run, float(lat.value)


def pb_server_stats_get(sv) -> pb_server_stats:
    s = pb_server_stats()
    _check(load().pb_server_stats_get(sv, ctypes.byref(s)))
    return s


def pb_server_destroy(sv):
    if sv:
        load().pb_server_destroy(sv)


# ------------------------------------------------------- convenience layer
def anneal(topo: int, J: np.ndarray, betas_or_sched, replicas: int, seed: int, h=None, L: int = 0, n: int = 0,
           form: int = PB_FORM_AUTO, target_energy: float = math.nan, stream=None) -> dict:
    """Create the instance, run one anneal, read every result back (synchronous)."""
    inst = pb_create_instance(topo, J, h, None, L=L, n=n, stream=stream)
    try:
        sched = betas_or_sched
        if not isinstance(sched, pb_schedule):
            b = np.asarray(betas_or_sched, dtype=np.float64)
            sched = make_schedule(PB_SCHED_EXPLICIT, b.size, betas=b)
        run = pb_anneal(inst, sched, replicas, seed, make_opts(form, target_energy), stream=stream)
        try:
            N = pb_instance_spins(inst)
            fe, be, bs = pb_energy(run, replicas)
            return dict(final_E=fe, best_E=be, best_sweep=bs, final_state=pb_final_states(run, replicas, N),
                        best_state=pb_best_states(run, replicas, N), target_sweep=pb_target_sweeps(run, replicas),
                        device_ms=pb_run_device_ms(run))
        finally:
            pb_run_destroy(run)
    finally:
        pb_instance_destroy(inst)

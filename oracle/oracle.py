"""Python face of the plain CPU oracle (``pbit_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline / reference arm may import this module.  The CUDA
library and its Python binding never do.

The C file is compiled with gcc on first use into ``oracle/_build``.  All
arrays cross as numpy arrays; couplings and fields are FP64.

What each function follows in the paper (arXiv 2510.23419):
  energy            Eq. 1 (sign: E = -sum J m m - sum h m, so that Eq. 2/3 sample exp(-beta E))
  fields            Eq. 3 with the field term, F_i = sum_j J_ij m_j + h_i
  threshold         Eq. 2 p-bit, uint32 threshold reading (see the C file)
  schedule          Sec. 1.3.1 classical annealing, Algorithm 1's linear beta step
  anneal            Sec. 1.2.2 update groups + Sec. 1.3.1 classical annealing
  class_step        one update-group step of that loop, from given states
  gen_ea/gen_biclique  Sec. 2 random cubic lattices / Sec. 3 random bicliques
  brute_force       exhaustive enumeration (Boltzmann law of Sec. 1.2.1)

Parity pins live in ``tests/test_oracle_*.py``; no function here is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIST_PM1, DIST_GAUSS, DIST_UNIF = 0, 1, 2
SCHED_LINEAR, SCHED_GEOMETRIC, SCHED_EXPLICIT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u32, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            lib.orc_philox_many.argtypes = [i64, P, P, P]
            lib.orc_rand_word.argtypes = [u64, u32, u32, u32, u32, ctypes.c_int]
            lib.orc_rand_word.restype = u32
            lib.orc_coupling.argtypes = [ctypes.c_int, u64, i64]
            lib.orc_coupling.restype = f64
            lib.orc_gen_ea.argtypes = [i32, i32, u64, P]
            lib.orc_gen_biclique.argtypes = [i32, i32, u64, P]
            lib.orc_ea_edges.argtypes = [i32, P, P]
            lib.orc_ea_colour.argtypes = [i32, P]
            lib.orc_biclique_edges.argtypes = [i32, P, P]
            lib.orc_biclique_colour.argtypes = [i32, P]
            lib.orc_count_monochrome.argtypes = [i64, P, P, P]
            lib.orc_count_monochrome.restype = i64
            lib.orc_energy.argtypes = [i32, i64, P, P, P, P, P]
            lib.orc_energy.restype = f64
            lib.orc_brute_force.argtypes = [i32, i64, P, P, P, P, P]
            lib.orc_brute_force.restype = ctypes.c_int
            lib.orc_schedule.argtypes = [i32, f64, f64, i32, i32, P, P]
            lib.orc_schedule.restype = ctypes.c_int
            lib.orc_threshold.argtypes = [f64, f64]
            lib.orc_threshold.restype = u32
            lib.orc_fields.argtypes = [i32, i64, P, P, P, P, P, P]
            lib.orc_anneal.argtypes = [i32, i64, P, P, P, P, P, i32, P, i32, i32, i32, u64,
                                       P, P, P, P, P, P, P]
            lib.orc_anneal.restype = ctypes.c_int
            lib.orc_class_step.argtypes = [i32, i64, P, P, P, P, P, i32, i32, f64, i32, i32, i32, u64, P, P, P]
            lib.orc_class_step.restype = ctypes.c_int
            lib.orc_pt.argtypes = [i32, i64, P, P, P, P, P, i32, P, i32, i32, i32, u64, P, P, P, P, P, P, P]
            lib.orc_pt.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- RNG
def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of n counters ([n,4] uint32) under n keys ([n,2] uint32) -> [n,4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    assert ctr.shape[0] == key.shape[0]
    out = np.empty_like(ctr)
    _load().orc_philox_many(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


def rand_word(seed: int, c0: int, c1: int, c2: int, c3: int, idx: int) -> int:
    return int(_load().orc_rand_word(seed, c0, c1, c2, c3, idx))


# ----------------------------------------------------------- instances
def gen_ea(L: int, dist: int, seed: int) -> np.ndarray:
    """Random EA couplings, [3, L^3] float64: bond (d, i) joins site i to its +x/+y/+z neighbour."""
    J = np.empty((3, L ** 3), dtype=np.float64)
    _load().orc_gen_ea(L, dist, seed, _p(J))
    return J


def gen_biclique(n: int, dist: int, seed: int) -> np.ndarray:
    """Random biclique couplings, [n, n] float64: J[i, j] joins left i to right j."""
    J = np.empty((n, n), dtype=np.float64)
    _load().orc_gen_biclique(n, dist, seed, _p(J))
    return J


def ea_graph(L: int):
    """Edge list (eu, ev) of the periodic L^3 lattice in bond order (d, i), and the checkerboard colours."""
    N = L ** 3
    eu = np.empty(3 * N, dtype=np.int32)
    ev = np.empty(3 * N, dtype=np.int32)
    col = np.empty(N, dtype=np.int32)
    lib = _load()
    lib.orc_ea_edges(L, _p(eu), _p(ev))
    lib.orc_ea_colour(L, _p(col))
    return eu, ev, col


def biclique_graph(n: int):
    """Edge list of K_{n,n} in bond order (i, j) (right spins are n..2n-1), and the side colours."""
    eu = np.empty(n * n, dtype=np.int32)
    ev = np.empty(n * n, dtype=np.int32)
    col = np.empty(2 * n, dtype=np.int32)
    lib = _load()
    lib.orc_biclique_edges(n, _p(eu), _p(ev))
    lib.orc_biclique_colour(n, _p(col))
    return eu, ev, col


def count_monochrome(eu, ev, colour) -> int:
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    colour = np.ascontiguousarray(colour, np.int32)
    return int(_load().orc_count_monochrome(eu.size, _p(eu), _p(ev), _p(colour)))


# -------------------------------------------------------------- energies
def _h(h, N):
    return None if h is None else np.ascontiguousarray(h, dtype=np.float64).reshape(N)


def energy(eu, ev, J, h, m) -> float:
    m = np.ascontiguousarray(m, dtype=np.int8)
    N = m.size
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    hh = _h(h, N)
    return float(_load().orc_energy(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(m)))


def fields(eu, ev, J, h, m) -> np.ndarray:
    m = np.ascontiguousarray(m, dtype=np.int8)
    N = m.size
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    hh = _h(h, N)
    F = np.empty(N, dtype=np.float64)
    _load().orc_fields(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(m), _p(F))
    return F


def brute_force(N: int, eu, ev, J, h=None) -> np.ndarray:
    """Energies of all 2^N states; bit i of the index set <=> m_i = +1."""
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    hh = _h(h, N)
    out = np.empty(1 << N, dtype=np.float64)
    rc = _load().orc_brute_force(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(out))
    if rc != 0:
        raise ValueError(f"brute force failed ({rc})")
    return out


def state_from_index(N: int, idx: int) -> np.ndarray:
    return np.array([1 if (idx >> i) & 1 else -1 for i in range(N)], dtype=np.int8)


# ------------------------------------------------------ schedule / p-bit
def schedule(kind: int, beta0: float, beta1: float, S: int, step_duration: int = 1, betas=None) -> np.ndarray:
    out = np.empty(S, dtype=np.float64)
    ex = None if betas is None else np.ascontiguousarray(betas, dtype=np.float64)
    rc = _load().orc_schedule(kind, beta0, beta1, S, step_duration, _p(ex), _p(out))
    if rc != 0:
        raise ValueError("bad schedule")
    return out


def threshold(beta: float, F: float) -> int:
    return int(_load().orc_threshold(float(beta), float(F)))


# --------------------------------------------------------------- anneal
def anneal(eu, ev, J, h, colour, betas, R: int, seed: int, n_colours: int | None = None,
           trace: bool = False, r_first: int = 0) -> dict:
    """Classical annealing of replicas r_first..r_first+R-1 (update groups in colour order); see the C file."""
    colour = np.ascontiguousarray(colour, np.int32)
    N = colour.size
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    assert J.size == eu.size == ev.size
    hh = _h(h, N)
    betas = np.ascontiguousarray(betas, np.float64)
    S = betas.size
    if n_colours is None:
        n_colours = int(colour.max()) + 1 if N else 1
    out = dict(
        final_E=np.empty(R, np.float64), best_E=np.empty(R, np.float64), best_sweep=np.empty(R, np.int32),
        final_state=np.empty((R, N), np.int8), best_state=np.empty((R, N), np.int8),
    )
    tr = np.empty((R, S), np.float64) if trace else None
    err = ctypes.c_double(0.0)
    rc = _load().orc_anneal(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(colour), n_colours, _p(betas), S, r_first,
                            R, seed, _p(out["final_E"]), _p(out["best_E"]), _p(out["best_sweep"]),
                            _p(out["final_state"]), _p(out["best_state"]), _p(tr), ctypes.byref(err))
    if rc == -2:
        raise ValueError("colouring has an edge inside a colour class")
    if rc != 0:
        raise ValueError(f"oracle anneal failed ({rc})")
    out["max_incr_err"] = err.value
    if trace:
        out["trace_E"] = tr
    return out


def class_step(eu, ev, J, h, colour, c: int, beta: float, s: int, states, seed: int, r_first: int = 0,
               n_colours: int | None = None) -> dict:
    """One update-group step (Sec. 1.2.2) of sweep s at inverse temperature beta: colour class c of the
    given states ([R, N] int8 +-1; row r is replica r_first + r) takes its decisions, every other spin
    is kept.  Returns the new states, and per updated spin the FP64 probability P = 1/2 + tanh(beta F)/2
    and the decision word w (NaN / 0 elsewhere)."""
    colour = np.ascontiguousarray(colour, np.int32)
    N = colour.size
    m = np.array(states, dtype=np.int8, copy=True).reshape(-1, N)
    R = m.shape[0]
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    hh = _h(h, N)
    if n_colours is None:
        n_colours = int(colour.max()) + 1
    P = np.full((R, N), np.nan)
    w = np.zeros((R, N), np.uint32)
    rc = _load().orc_class_step(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(colour), n_colours, c, float(beta), s,
                                r_first, R, seed, _p(m), _p(P), _p(w))
    if rc == -2:
        raise ValueError("colouring has an edge inside a colour class")
    if rc != 0:
        raise ValueError(f"oracle class step failed ({rc})")
    return dict(state=m, P=P, w=w)


def anneal_ea(L: int, J, h, betas, R: int, seed: int, **kw) -> dict:
    if L < 2 or L % 2:
        raise ValueError("the checkerboard needs an even L >= 2")
    eu, ev, col = ea_graph(L)
    return anneal(eu, ev, np.asarray(J, np.float64).reshape(-1), h, col, betas, R, seed, 2, **kw)


def anneal_biclique(n: int, J, h, betas, R: int, seed: int, **kw) -> dict:
    eu, ev, col = biclique_graph(n)
    return anneal(eu, ev, np.asarray(J, np.float64).reshape(-1), h, col, betas, R, seed, 2, **kw)


# ------------------------------------------------ benchmarking protocol
def find_imin(eu, ev, J, h, colour, ground: float, p: float, p_succ: float, i_start: int, i_step: int,
              trials: int, beta_i: float, beta_f: float, i_max: int, seed: int, n_colours: int | None = None):
    """Algorithm 1 (Sec. 4.1.3) as printed: budgets i = i_start, i_start + i_step, ...; at each, run the
    trials one after another (trial j = replica j of seed + i), count fails (best energy > p G) and stop
    the budget early once the fails exceed m_max = round(t (1 - p_succ)) (half up); return the first budget that
    passes (None if none up to i_max).  One iteration = one colour-class step: ceil(i / k) sweeps with
    a linear schedule (both ends included)."""
    colour = np.ascontiguousarray(colour, np.int32)
    k = int(colour.max()) + 1 if n_colours is None else n_colours
    theta = p * ground
    m_max = int(np.floor(trials * (1.0 - p_succ) + 0.5))  # round half up
    i = i_start
    while i <= i_max:
        S = (i + k - 1) // k
        betas = schedule(SCHED_LINEAR, beta_i, beta_f, S)
        m = 0
        for j in range(trials):
            v = anneal(eu, ev, J, h, colour, betas, 1, seed + i, n_colours=k, r_first=j)["best_E"][0]
            if v > theta:
                m += 1
                if m > m_max:
                    break
        if m <= m_max:
            return i
        i += i_step
    return None


# ------------------------------------------------------- parallel tempering
def anneal_pt(eu, ev, J, h, colour, ladder, S: int, R: int, seed: int, n_colours: int | None = None) -> dict:
    """Parallel tempering (see the C file): per slot g = k R + r results, the final temperature index of
    every slot and the accepted exchanges per temperature pair."""
    colour = np.ascontiguousarray(colour, np.int32)
    N = colour.size
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    J = np.ascontiguousarray(J, np.float64).reshape(-1)
    hh = _h(h, N)
    ladder = np.ascontiguousarray(ladder, np.float64)
    M = ladder.size
    if n_colours is None:
        n_colours = int(colour.max()) + 1
    G = M * R
    out = dict(final_E=np.empty(G), best_E=np.empty(G), best_sweep=np.empty(G, np.int32),
               final_state=np.empty((G, N), np.int8), best_state=np.empty((G, N), np.int8),
               slot_temp=np.empty(G, np.int32), n_accept=np.zeros(max(M - 1, 1), np.int64))
    rc = _load().orc_pt(N, eu.size, _p(eu), _p(ev), _p(J), _p(hh), _p(colour), n_colours, _p(ladder), M, S, R, seed,
                        _p(out["final_E"]), _p(out["best_E"]), _p(out["best_sweep"]), _p(out["final_state"]),
                        _p(out["best_state"]), _p(out["slot_temp"]), _p(out["n_accept"]))
    if rc == -2:
        raise ValueError("colouring has an edge inside a colour class")
    if rc != 0:
        raise ValueError(f"oracle parallel tempering failed ({rc})")
    out["n_accept"] = out["n_accept"][: M - 1]
    return out

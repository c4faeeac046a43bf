"""Seeded synthetic inputs shared by the tests and the benchmark.

Only random draws live here (numpy's PCG64 generator): couplings with the laws
of the paper's random instances (Sec. 2: random cubic lattices; Sec. 3: random
bicliques with couplings from [-1, 1]), integer or real fields, and random
+-1 states.  No step of the annealing method is computed here.
"""
from __future__ import annotations

import numpy as np


def ea_couplings(L: int, law: str, seed: int) -> np.ndarray:
    """[3, L^3] bonds: 'pm1' -> int8 +-1 (fair coin), 'gauss' -> float32 N(0,1)."""
    rng = np.random.default_rng(seed)
    if law == "pm1":
        return rng.choice(np.array([-1, 1], np.int8), size=(3, L ** 3))
    if law == "gauss":
        return rng.standard_normal((3, L ** 3)).astype(np.float32)
    raise ValueError(law)


def biclique_couplings(n: int, law: str, seed: int) -> np.ndarray:
    """[n, n]: 'pm1' -> int8 +-1, 'gauss' -> float32 N(0,1), 'unif' -> float32 U(-1,1)."""
    rng = np.random.default_rng(seed)
    if law == "pm1":
        return rng.choice(np.array([-1, 1], np.int8), size=(n, n))
    if law == "gauss":
        return rng.standard_normal((n, n)).astype(np.float32)
    if law == "unif":
        return rng.uniform(-1, 1, (n, n)).astype(np.float32)
    raise ValueError(law)


def int_fields(N: int, hmax: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(-hmax, hmax + 1, size=N).astype(np.int8)


def real_fields(N: int, scale: float, seed: int) -> np.ndarray:
    return (scale * np.random.default_rng(seed).standard_normal(N)).astype(np.float32)


def states(R: int, N: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).choice(np.array([-1, 1], np.int8), size=(R, N))


# ---------------------------------------------------------------- graphs
# Edge lists (eu, ev) of the sparse test and bench topologies; each undirected
# edge once.  Structure only: no coupling values, no colouring.

def graph_periodic_cube(L: int):
    """Periodic L^3 lattice, 6 neighbours; odd L is not bipartite (3 colours)."""
    idx = np.arange(L ** 3).reshape(L, L, L)  # [z][y][x]
    eu, ev = [], []
    for ax in (2, 1, 0):
        eu.append(idx.reshape(-1))
        ev.append(np.roll(idx, -1, axis=ax).reshape(-1))
    return np.concatenate(eu).astype(np.int32), np.concatenate(ev).astype(np.int32)


def graph_king(Lx: int, Ly: int):
    """Open 2D king's graph (8 neighbours), chromatic number 4."""
    eu, ev = [], []
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            for dx, dy in ((1, 0), (0, 1), (1, 1), (-1, 1)):
                X, Y = x + dx, y + dy
                if 0 <= X < Lx and 0 <= Y < Ly:
                    eu.append(i)
                    ev.append(Y * Lx + X)
    return np.array(eu, np.int32), np.array(ev, np.int32)


def graph_random(N: int, n_edges: int, seed: int):
    """Random simple graph: n_edges distinct pairs, no self-loops."""
    rng = np.random.default_rng(seed)
    seen, eu, ev = set(), [], []
    while len(eu) < n_edges:
        u, v = (int(x) for x in rng.integers(0, N, size=2))
        if u == v or (min(u, v), max(u, v)) in seen:
            continue
        seen.add((min(u, v), max(u, v)))
        eu.append(u)
        ev.append(v)
    return np.array(eu, np.int32), np.array(ev, np.int32)


def edge_couplings(n_edges: int, law: str, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if law == "pm1":
        return np.where(rng.random(n_edges) < 0.5, 1, -1).astype(np.int8)
    if law == "gauss":
        return rng.normal(size=n_edges).astype(np.float32)
    return rng.uniform(-1.0, 1.0, size=n_edges).astype(np.float32)

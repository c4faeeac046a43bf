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

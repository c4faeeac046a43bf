"""The sparsified biclique (host only): every biclique edge appears once with its
coupling between copies of its two ends, copies of a vertex form a path of
ferromagnetic copy edges, no copy has more than six distinct neighbours, the
two colours are a proper colouring (checked with the oracle's own count), and
on states whose copies agree the copy graph's energy is the biclique's energy
minus copy_strength per copy edge (oracle energies of both graphs)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


@pytest.mark.parametrize("n,per,cs,law", [(8, 4, 2, "pm1"), (13, 3, 1, "pm1"), (16, 4, 3, "gauss"), (5, 1, 2, "pm1")])
def test_structure_and_energy(pb, orc, n, per, cs, law):
    rng = np.random.default_rng(n)
    if law == "pm1":
        J = np.where(rng.random((n, n)) < 0.5, 1, -1).astype(np.int8)
    else:
        J = rng.normal(size=(n, n)).astype(np.float32)
    sp = pb.pb_sparsify_biclique(J, per, cs)
    N, eu, ev, Js, col, cof = sp["N"], sp["eu"], sp["ev"], sp["J"], sp["colour"], sp["copy_of"]
    # original edges: the first n^2, in row-major order, between copies of i and j
    assert np.array_equal(cof[eu[: n * n]], np.repeat(np.arange(n), n))
    assert np.array_equal(cof[ev[: n * n]], n + np.tile(np.arange(n), n))
    assert np.array_equal(Js[: n * n].astype(np.float64), J.reshape(-1).astype(np.float64))
    # copy edges: consecutive ids of the same vertex, ferromagnetic
    ce_u, ce_v, ce_J = eu[n * n:], ev[n * n:], Js[n * n:].astype(np.float64)
    assert np.all(ce_v == ce_u + 1) and np.all(cof[ce_u] == cof[ce_v]) and np.all(ce_J > 0)
    strength = np.zeros(N)
    np.add.at(strength, ce_v, ce_J)
    first = np.r_[True, cof[1:] != cof[:-1]]
    assert np.all(strength[~first] == cs) and np.all(strength[first] == 0)
    # degree bound (distinct neighbours) and proper 2-colouring
    nb = [set() for _ in range(N)]
    for u, v in zip(eu, ev):
        nb[u].add(v)
        nb[v].add(u)
    assert max(len(s) for s in nb) <= per + 2 <= 6
    assert orc.count_monochrome(eu, ev, col) == 0 and set(col.tolist()) <= {0, 1}
    # energy of agreeing copies
    beu, bev, _ = orc.biclique_graph(n)
    m = rng.choice(np.array([-1, 1], np.int8), size=2 * n)
    ms = m[cof]
    e_orig = orc.energy(beu, bev, J.reshape(-1).astype(np.float64), None, m)
    e_sp = orc.energy(eu, ev, Js.astype(np.float64), None, ms)
    assert abs(e_sp - (e_orig - cs * (N - 2 * n))) <= 1e-9 * max(1.0, abs(e_orig))
    # projection recovers m from agreeing copies, and majority otherwise
    assert np.array_equal(pb.pb_sparse_project(cof, 2 * n, ms[None, :])[0], m)
    flip = ms.copy()
    flip[first.nonzero()[0]] *= -1  # flip copy 0 of every vertex with >= 3 copies: majority unchanged
    counts = np.bincount(cof, minlength=2 * n)
    proj = pb.pb_sparse_project(cof, 2 * n, flip[None, :])[0]
    many = counts >= 3
    assert np.array_equal(proj[many], m[many])

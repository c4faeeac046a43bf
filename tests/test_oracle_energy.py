"""Pins for the oracle's energy (Eq. 1) and local fields (Eq. 3).

Checked against what the mathematics fixes, not against the oracle's own
formula: closed-form ground states (ferromagnets, a planted Mattis instance),
exhaustive enumeration, global spin-flip symmetry, the flip identity of Eq. 3
(the energy change of a single flip equals 2 m_i F_i) and independent numpy
restatements (np.roll on the periodic cube, a matrix product for bicliques).
"""
import numpy as np
import pytest


def test_single_bond_sign(orc):
    # Eq. 1 with the reading E = -J m1 m2 (a positive coupling favours alignment)
    eu = np.array([0], np.int32); ev = np.array([1], np.int32)
    for J in (1.0, -1.0, 0.37):
        for m1 in (1, -1):
            for m2 in (1, -1):
                E = orc.energy(eu, ev, np.array([J]), None, np.array([m1, m2], np.int8))
                assert E == pytest.approx(-J * m1 * m2, abs=0)
    # field term: E = -h m
    E = orc.energy(eu, ev, np.array([0.0]), np.array([0.5, -2.0]), np.array([1, 1], np.int8))
    assert E == pytest.approx(-(0.5 - 2.0))


@pytest.mark.parametrize("L", [2, 4, 6])
def test_ea_ferromagnet_closed_form(orc, L):
    N = L ** 3
    eu, ev, col = orc.ea_graph(L)
    J = np.ones(3 * N)
    assert orc.energy(eu, ev, J, None, np.ones(N, np.int8)) == -3 * N
    assert orc.energy(eu, ev, J, None, -np.ones(N, np.int8)) == -3 * N
    # the checkerboard state breaks every bond
    m = np.where(col == 0, 1, -1).astype(np.int8)
    assert orc.energy(eu, ev, J, None, m) == 3 * N


def test_ea_ferromagnet_brute_force(orc):
    # L=2: 8 sites, 24 bonds (double bonds kept); exactly two ground states at -24
    eu, ev, col = orc.ea_graph(2)
    E = orc.brute_force(8, eu, ev, np.ones(24))
    assert E.min() == -24
    assert set(np.nonzero(E == E.min())[0].tolist()) == {0, 255}


@pytest.mark.parametrize("n", [3, 5, 8])
def test_biclique_ferromagnet_brute_force(orc, n):
    # all-ferromagnetic K_{n,n}: E0 = -n^2 with the two uniform states only
    eu, ev, col = orc.biclique_graph(n)
    E = orc.brute_force(2 * n, eu, ev, np.ones(n * n))
    assert E.min() == -n * n
    assert set(np.nonzero(E == E.min())[0].tolist()) == {0, (1 << 2 * n) - 1}


def test_mattis_planted(orc):
    # J_ij = xi_i xi_j is a gauge transform of the ferromagnet: ground states +-xi at -#edges
    rng = np.random.default_rng(5)
    L = 4; N = L ** 3
    eu, ev, col = orc.ea_graph(L)
    xi = rng.choice([-1, 1], size=N).astype(np.int8)
    J = (xi[eu].astype(np.float64) * xi[ev])
    assert orc.energy(eu, ev, J, None, xi) == -3 * N
    assert orc.energy(eu, ev, J, None, -xi) == -3 * N
    for _ in range(20):
        m = xi.copy(); flip = rng.integers(0, N, size=rng.integers(1, 5)); m[flip] *= -1
        assert orc.energy(eu, ev, J, None, m) > -3 * N


def test_global_flip(orc):
    rng = np.random.default_rng(7)
    eu, ev, col = orc.ea_graph(4)
    J = rng.normal(size=eu.size)
    h = rng.normal(size=64)
    for _ in range(10):
        m = rng.choice([-1, 1], size=64).astype(np.int8)
        e0 = orc.energy(eu, ev, J, None, m)
        assert orc.energy(eu, ev, J, None, -m) == pytest.approx(e0, rel=1e-13, abs=1e-12)
        # with a field the flip changes E by 2 sum h m
        e1 = orc.energy(eu, ev, J, h, m)
        assert orc.energy(eu, ev, J, h, -m) == pytest.approx(e1 + 2 * np.dot(h, m), rel=1e-12, abs=1e-12)


def test_ea_energy_numpy_roll(orc):
    # independent restatement on the periodic cube: bond d of site (x,y,z) meets the site one step along axis d
    rng = np.random.default_rng(11)
    L = 6; N = L ** 3
    eu, ev, col = orc.ea_graph(L)
    J = rng.normal(size=(3, N))
    h = rng.normal(size=N)
    m = rng.choice([-1, 1], size=N).astype(np.int8)
    m3 = m.reshape(L, L, L).astype(np.float64)           # index [z, y, x]
    E = 0.0
    for d, axis in ((0, 2), (1, 1), (2, 0)):
        E -= np.sum(J[d].reshape(L, L, L) * m3 * np.roll(m3, -1, axis=axis))
    E -= np.dot(h, m)
    assert orc.energy(eu, ev, J, h, m) == pytest.approx(E, rel=1e-12)


def test_biclique_energy_matrix_form(orc):
    rng = np.random.default_rng(13)
    n = 9
    eu, ev, col = orc.biclique_graph(n)
    J = rng.normal(size=(n, n))
    h = rng.normal(size=2 * n)
    m = rng.choice([-1, 1], size=2 * n).astype(np.int8)
    a, b = m[:n].astype(float), m[n:].astype(float)
    E = -a @ J @ b - h @ m
    assert orc.energy(eu, ev, J, h, m) == pytest.approx(E, rel=1e-12)


@pytest.mark.parametrize("topo", ["ea", "biclique"])
def test_flip_identity_eq3(orc, topo):
    # Eq. 3: flipping spin i changes E by 2 m_i F_i, F_i = sum_j J_ij m_j + h_i
    rng = np.random.default_rng(17)
    if topo == "ea":
        eu, ev, col = orc.ea_graph(4); N = 64
    else:
        eu, ev, col = orc.biclique_graph(7); N = 14
    J = rng.normal(size=eu.size)
    h = rng.normal(size=N)
    m = rng.choice([-1, 1], size=N).astype(np.int8)
    F = orc.fields(eu, ev, J, h, m)
    E0 = orc.energy(eu, ev, J, h, m)
    for i in range(N):
        mm = m.copy(); mm[i] = -mm[i]
        assert orc.energy(eu, ev, J, h, mm) - E0 == pytest.approx(2 * m[i] * F[i], rel=1e-10, abs=1e-10)


def test_colourings_proper(orc):
    for L in (2, 4, 6, 8):
        eu, ev, col = orc.ea_graph(L)
        assert orc.count_monochrome(eu, ev, col) == 0
        assert (col == 0).sum() == (col == 1).sum() == L ** 3 // 2
    eu, ev, col = orc.biclique_graph(6)
    assert orc.count_monochrome(eu, ev, col) == 0
    # odd L: the periodic cube is not bipartite, the checkerboard has internal edges
    eu, ev, col = orc.ea_graph(3)
    assert orc.count_monochrome(eu, ev, col) > 0

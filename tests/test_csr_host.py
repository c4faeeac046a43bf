"""Host side of general sparse instances (no GPU): the greedy colouring is a
proper colouring (no edge inside a class, checked with the oracle's own count),
uses at most max degree + 1 colours, is deterministic, meets the known
chromatic numbers of small graphs, and rejects invalid edge lists."""
import numpy as np
import pytest

import synth_inputs as syn


@pytest.fixture(scope="module")
def pb():
    from paper_2510_23419_gb300 import _build, native
    _build.build()
    native.load()
    return native


def _degrees(N, eu, ev):
    return np.bincount(np.concatenate([eu, ev]), minlength=N)


@pytest.mark.parametrize("name", ["cube5", "cube4", "king", "random", "dense"])
def test_greedy_is_proper(pb, orc, name):
    N, (eu, ev) = {
        "cube5": (125, syn.graph_periodic_cube(5)),
        "cube4": (64, syn.graph_periodic_cube(4)),
        "king": (63, syn.graph_king(9, 7)),
        "random": (400, syn.graph_random(400, 1600, 5)),
        "dense": (60, syn.graph_random(60, 1200, 6)),
    }[name]
    col, k = pb.pb_greedy_colouring(N, eu, ev)
    assert orc.count_monochrome(eu, ev, col) == 0
    assert col.min() == 0 and col.max() == k - 1
    assert k <= _degrees(N, eu, ev).max() + 1
    col2, k2 = pb.pb_greedy_colouring(N, eu, ev)
    assert k2 == k and np.array_equal(col, col2)


def test_known_chromatic_numbers(pb):
    # odd cycle: 3; complete graph K_5: 5; no edges: 1; even cycle: 2
    c7 = (np.arange(7), (np.arange(7) + 1) % 7)
    assert pb.pb_greedy_colouring(7, *c7)[1] == 3
    iu = np.array([i for i in range(5) for j in range(i + 1, 5)])
    iv = np.array([j for i in range(5) for j in range(i + 1, 5)])
    assert pb.pb_greedy_colouring(5, iu, iv)[1] == 5
    assert pb.pb_greedy_colouring(4, np.zeros(0, np.int32), np.zeros(0, np.int32))[1] == 1
    c8 = (np.arange(8), (np.arange(8) + 1) % 8)
    assert pb.pb_greedy_colouring(8, *c8)[1] == 2


def test_invalid_edges_rejected(pb):
    with pytest.raises(pb.PbError):
        pb.pb_greedy_colouring(4, np.array([0, 1]), np.array([1, 1]))  # self-loop
    with pytest.raises(pb.PbError):
        pb.pb_greedy_colouring(4, np.array([0]), np.array([4]))  # out of range

"""Pins for the oracle's annealing schedule (Sec. 1.3.1; Algorithm 1's linear
beta step; the conclusion's linear 0.35 -> 3.5 schedule).  Closed forms: end
points, constant steps (linear) or ratios (geometric), step durations."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_protocol.json")


def test_linear_endpoints_and_steps(orc):
    with open(GOLDEN) as f:
        g = json.load(f)
    b0, b1 = g["linear_schedule"]["beta_initial"], g["linear_schedule"]["beta_final"]
    S = 1000
    b = orc.schedule(orc.SCHED_LINEAR, b0, b1, S)
    assert b[0] == b0 and b[-1] == pytest.approx(b1, rel=1e-15)
    d = np.diff(b)
    assert np.allclose(d, (b1 - b0) / (S - 1), rtol=1e-9)


def test_geometric(orc):
    b = orc.schedule(orc.SCHED_GEOMETRIC, 0.1, 5.0, 101)
    assert b[0] == 0.1 and b[-1] == pytest.approx(5.0, rel=1e-14)
    r = b[1:] / b[:-1]
    assert np.allclose(r, 50.0 ** (1 / 100), rtol=1e-12)


def test_step_duration(orc):
    b = orc.schedule(orc.SCHED_LINEAR, 1.0, 2.0, 10, step_duration=3)   # levels 0..3 (ceil(10/3)=4)
    assert np.allclose(b, [1, 1, 1, 4 / 3, 4 / 3, 4 / 3, 5 / 3, 5 / 3, 5 / 3, 2])
    one = orc.schedule(orc.SCHED_LINEAR, 0.4, 9.0, 5, step_duration=5)
    assert np.all(one == 0.4)


def test_explicit(orc):
    x = np.array([0.3, 0.1, 2.0])
    assert np.array_equal(orc.schedule(orc.SCHED_EXPLICIT, 0, 0, 3, betas=x), x)

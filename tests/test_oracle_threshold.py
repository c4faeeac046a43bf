"""Pins for the oracle's p-bit threshold (Eq. 2, uint32 reading).

T(beta, F) = min(floor((1/2 + tanh(beta F)/2) 2^32), 2^32 - 1).  Checked
against the exact value from 60-digit arithmetic (mpmath, through the logistic
identity 1/2 + tanh(x)/2 = 1 / (1 + e^{-2x})), the special value beta = 0,
odd symmetry, monotonicity and saturation.
"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")


def _exact(beta, F):
    mpmath.mp.dps = 60
    x = mpmath.mpf(beta) * mpmath.mpf(F)
    P = 1 / (1 + mpmath.e ** (-2 * x))
    return int(mpmath.floor(P * 2 ** 32))


def test_threshold_beta_zero(orc):
    for F in (-6, -1, 0, 3, 2.5):
        assert orc.threshold(0.0, F) == 2 ** 31


def test_threshold_against_high_precision(orc):
    rng = np.random.default_rng(3)
    cases = [(b, F) for b in (0.1, 0.35, 1.0, 3.5, 5.0) for F in range(-12, 13)]
    cases += [(float(b), float(F)) for b, F in zip(rng.uniform(0, 5, 200), rng.normal(0, 3, 200))]
    for b, F in cases:
        ex = min(_exact(b, F), 2 ** 32 - 1)
        assert abs(orc.threshold(b, F) - ex) <= 1, (b, F)


def test_threshold_odd_monotone_saturating(orc):
    for b in (0.1, 0.7, 2.0, 5.0):
        Ts = [orc.threshold(b, F) for F in range(-20, 21)]
        assert all(x <= y for x, y in zip(Ts, Ts[1:]))
        for F in range(0, 21):
            s = orc.threshold(b, F) + orc.threshold(b, -F)
            assert 2 ** 32 - 2 <= s <= 2 ** 32
    assert orc.threshold(50.0, 6) == 2 ** 32 - 1
    assert orc.threshold(50.0, -6) == 0

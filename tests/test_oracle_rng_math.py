"""Pins of the oracle's random numbers and elementary functions.

Philox4x32-10 against the published known-answer vectors; the oracle's own
exp and ln against libm and mpmath (2 ulp); the type-7 quantile against numpy.
"""
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(orc.philox(ctr, key)) == want


def test_draw_uses_counter_blocks(orc):
    # draws 4q..4q+3 of one ant are the four words of one Philox block
    seed = 0x1234_5678_9abc_def0
    for t, a, q in [(0, 0, 0), (3, 7, 11), (199, 63, 2499)]:
        blk = orc.philox([q, a, t, 0], [seed & 0xffffffff, seed >> 32])
        assert [orc.draw(seed, t, a, 4 * q + w) for w in range(4)] == list(blk)


def _ulp_diff(a, b):
    ia = np.frombuffer(np.float64(a).tobytes(), np.int64)[0]
    ib = np.frombuffer(np.float64(b).tobytes(), np.int64)[0]
    return abs(int(ia) - int(ib))


def test_exp_within_two_ulp(orc):
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-50, 35, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                         [0.0, 1.0, -1.0, 0.5, 30.0, math.log(2), -math.log(2) / 2]])
    worst = max(_ulp_diff(orc.exp(x), math.exp(x)) for x in xs)
    assert worst <= 2
    assert orc.exp(0.0) == 1.0


def test_exp_against_mpmath(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    for x in [-37.25, -2.0, 0.125, 1.0, 7.5, 29.999]:
        ref = float(mpmath.exp(mpmath.mpf(x)))
        assert _ulp_diff(orc.exp(x), ref) <= 2


def test_ln_within_two_ulp(orc):
    rng = np.random.default_rng(6)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 20000)), 1.0 + rng.uniform(-1e-3, 1e-3, 2000),
                         rng.uniform(1.0, 1e9, 5000), [2.0, 0.5, 10.0, 1.0 + 2 ** -52, 1e9, 1581.0]])
    worst = max(_ulp_diff(orc.ln(x), math.log(x)) for x in xs if x != 1.0)
    assert worst <= 2
    assert orc.ln(1.0) == 0.0
    for k in (-40, -1, 1, 3, 60):
        assert abs(orc.ln(2.0 ** k) - k * math.log(2)) <= 2 * abs(k) * 2 ** -52


def test_ln_exp_roundtrip(orc):
    for x in np.linspace(-30, 30, 241):
        assert abs(orc.ln(orc.exp(x)) - x) <= 4e-15 * max(1.0, abs(x))


def test_quantile7_matches_numpy_linear(orc):
    rng = np.random.default_rng(7)
    for N in (1, 2, 3, 10, 11, 999, 1000, 12345):
        x = np.sort(rng.exponential(0.5, N))
        for q in (0.0, 0.5, 0.9, 0.99, 1.0):
            ref = np.quantile(x, q, method="linear")
            assert orc.quantile7(x, q) == pytest.approx(ref, rel=1e-14, abs=0)
    assert orc.quantile7(np.zeros(0), 0.9) == 0.0

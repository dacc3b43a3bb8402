"""Host logic of the benchmark's equal-error pairs (bench.py): the plain partner of an
adaptive error, the fallback closest pair, and the log-log interpolation of the plain
time at the adaptive error.  Plain runs: {fixed sweeps: (err, ms)}; adaptive runs:
[(TOL, err, ms)]."""

import numpy as np
import pytest

import bench

PLAIN = {1: (6.3e-4, 86.8), 2: (1.3e-5, 172.8), 3: (3.0e-7, 267.8), 4: (7.4e-9, 373.5),
         5: (2.5e-10, 486.1)}


def test_partner_is_the_fewest_sweeps_within_1_1x():
    assert bench.plain_partner(PLAIN, 3.0e-7) == 3          # equal error
    assert bench.plain_partner(PLAIN, 2.8e-7) == 3          # 3.0e-7 <= 1.1 * 2.8e-7
    assert bench.plain_partner(PLAIN, 2.5e-7) == 4          # 3.0e-7 > 1.1 * 2.5e-7
    assert bench.plain_partner(PLAIN, 1e-3) == 1
    assert bench.plain_partner(PLAIN, 1e-12) == 5           # none within: the most sweeps


def test_closest_pair_in_log():
    adapt = [(1e-5, 3.8e-7, 127.0), (5e-6, 3.6e-7, 154.0)]
    assert bench.closest_pair(PLAIN, adapt) == (1, 3)       # 3.6e-7 is closest to 3.0e-7
    adapt = [(1e-5, 1.0e-8, 100.0)]
    assert bench.closest_pair(PLAIN, adapt) == (0, 4)


def test_interpolation_is_exact_on_a_power_law_and_none_outside():
    # ms = 10 err^-0.25 on both points: the interpolant reproduces it in between
    plain = {1: (1e-4, 10 * 1e-4 ** -0.25), 2: (1e-8, 10 * 1e-8 ** -0.25)}
    for e in (1e-5, 3e-7, 1e-8, 1e-4):
        assert bench.interp_plain_ms(plain, e) == pytest.approx(10 * e ** -0.25, rel=1e-12)
    assert bench.interp_plain_ms(plain, 1e-3) is None
    assert bench.interp_plain_ms(plain, 1e-9) is None
    # the measured W2 scan: between 2 and 3 sweeps
    ms = bench.interp_plain_ms(PLAIN, 3.649e-7)
    assert 172.8 < ms < 267.8 and ms == pytest.approx(261.77, rel=1e-3)

"""Pins of the oracle's primitive pieces against published or closed-form values."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O


def test_philox_known_answers(golden_dir):
    """Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_series_log_matches_libm():
    """The deterministic logarithm of the shift update agrees with log() to a few ulp
    (relative) or 4e-17 (absolute, near x = 1 where log x is small)."""
    rng = np.random.default_rng(7)
    xs = np.concatenate([np.exp(rng.uniform(-20, 20, 4000)), 1.0 + rng.uniform(-0.05, 0.05, 4000),
                         [1.0, 2.0, 0.5, 1024.0, 1 / 3, math.sqrt(2), math.nextafter(math.sqrt(2), 2)]])
    for x in xs:
        a, b = O.series_log(float(x)), math.log(float(x))
        assert abs(a - b) <= 4 * math.ulp(b) + 4e-17, (x, a, b)
    assert O.series_log(1.0) == 0.0
    assert O.series_log(2.0 ** 10) == 10 * 0.6931471805599453


def test_series_log_nonpositive_is_zero():
    assert O.series_log(0.0) == 0.0
    assert O.series_log(-3.0) == 0.0

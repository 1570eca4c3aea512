"""Blocking analysis against closed forms."""
import math

import numpy as np

from oracle import blocking as Bk


def test_level_zero_is_plain_standard_error():
    rng = np.random.default_rng(1)
    x = rng.integers(-1000, 1000, 4096)
    lv = Bk.ratio_levels(x)
    assert lv[0][0] == 4096
    assert abs(lv[0][1] - x.mean()) < 1e-12
    assert abs(lv[0][2] - np.std(x, ddof=1) / math.sqrt(len(x))) < 1e-9 * lv[0][2]


def test_moments_are_exact_block_sums():
    x = np.arange(1, 17)
    lv = Bk.level_moments(x)
    assert [l["n"] for l in lv] == [16, 8, 4, 2, 1]
    assert lv[2]["sx"] == sum(range(1, 17)) and lv[2]["sxx"] == 10 ** 2 + 26 ** 2 + 42 ** 2 + 58 ** 2


def test_ar1_blocked_error_matches_closed_form():
    """AR(1) x_t = phi x_{t-1} + e_t: Var(mean) -> sigma^2 / ((1 - phi)^2 n)."""
    rng = np.random.default_rng(12)
    phi, sigma, n = 0.9, 1.0, 1 << 18
    e = rng.normal(0.0, sigma, n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - phi ** 2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    xi = np.round(x * 1e6).astype(np.int64)
    _, err, lvl = Bk.blocked_mean(xi)
    exact = sigma / (1 - phi) / math.sqrt(n) * 1e6
    assert lvl is not None and lvl >= 4
    assert abs(err / exact - 1) < 0.25, (err, exact)


def test_ratio_of_constant_denominator_matches_mean():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 100, 1024)
    y = np.full(1024, 7)
    lv_r = Bk.ratio_levels(x, y)
    lv_m = Bk.ratio_levels(x)
    for (n1, r1, e1), (n2, r2, e2) in zip(lv_r, lv_m):
        if n1 < 2:
            continue
        assert n1 == n2 and abs(r1 * 7 - r2) < 1e-12 and abs(e1 * 7 - e2) < 1e-9 * max(e2, 1e-30)

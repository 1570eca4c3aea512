"""Blocking analysis of the estimator time series -- TEST INFRASTRUCTURE ONLY.

The paper estimates a steady-state observable as the ratio of the time
averages of the numerator sum_ij rho_ij O_ji and of the trace (Sec. III.A); it
gives no error-bar method.  This module takes the reading used throughout
the project: Flyvbjerg-Petersen blocking (J. Chem. Phys. 91, 461 (1989)) of
numerator and denominator together, with the delta-method variance of the
ratio built from the block covariance, and a plateau chosen as the first
level k whose error e_k is not exceeded by the error e_q of any coarser level
with at least MIN_BLOCKS blocks by more than twice their combined
uncertainty, 2 sqrt(de_k^2 + de_q^2), where de = e / sqrt(2 (n - 1)).

Block sums are integers, so every moment below is exact (Python integers);
only the final combination is a floating-point division.
"""
from __future__ import annotations

import math
from fractions import Fraction

MIN_BLOCKS = 16


def level_moments(x, y=None):
    """Per level l (block length 2^l, blocks counted from the first sample):
    n, sum X, sum X^2, sum X*Y, sum Y, sum Y^2 over the complete block sums."""
    xs = [int(v) for v in x]
    ys = [1] * len(xs) if y is None else [int(v) for v in y]
    levels = []
    while len(xs) >= 1:
        n = len(xs)
        levels.append(dict(n=n, sx=sum(xs), sxx=sum(v * v for v in xs),
                           sxy=sum(a * b for a, b in zip(xs, ys)), sy=sum(ys),
                           syy=sum(v * v for v in ys)))
        if n < 2:
            break
        m = n // 2
        xs = [xs[2 * k] + xs[2 * k + 1] for k in range(m)]
        ys = [ys[2 * k] + ys[2 * k + 1] for k in range(m)]
    return levels


def ratio_variance(lv):
    """Delta-method variance of R = sum X / sum Y from one level's moments:
    [A SY^2 - 2 SX SY C + SX^2 D] / ((n-1) SY^4), with A = n SXX - SX^2,
    C = n SXY - SX SY, D = n SYY - SY^2 (all exact integers)."""
    n, sx, sy = lv["n"], lv["sx"], lv["sy"]
    if n < 2 or sy == 0:
        return float("nan")
    A = n * lv["sxx"] - sx * sx
    Cc = n * lv["sxy"] - sx * sy
    D = n * lv["syy"] - sy * sy
    num = A * sy * sy - 2 * sx * sy * Cc + sx * sx * D
    den = (n - 1) * sy ** 4
    return float(Fraction(num, den))


def ratio_levels(x, y=None):
    """[(n_blocks, R_l, stderr_l)] per level."""
    out = []
    for lv in level_moments(x, y):
        var = ratio_variance(lv)
        err = math.sqrt(var) if var == var and var >= 0 else float("nan")
        R = lv["sx"] / lv["sy"] if lv["sy"] != 0 else float("nan")
        out.append((lv["n"], R, err))
    return out


def plateau(levels, min_blocks=MIN_BLOCKS):
    """Index of the plateau level, or None if no level has enough blocks."""
    valid = [k for k, (n, _, e) in enumerate(levels) if n >= min_blocks and e == e]
    if not valid:
        return None
    def de(q):
        n, _, e = levels[q]
        return e / math.sqrt(2.0 * (n - 1))

    for k in valid:
        e = levels[k][2]
        if all(levels[q][2] <= e + 2.0 * math.sqrt(de(k) ** 2 + de(q) ** 2) for q in valid if q > k):
            return k
    return valid[-1]


def blocked_ratio(x, y=None, min_blocks=MIN_BLOCKS):
    """(R over all samples, blocked stderr, plateau level)."""
    lv = ratio_levels(x, y)
    k = plateau(lv, min_blocks)
    R = lv[0][1]
    if k is None:
        return R, float("nan"), None
    return R, lv[k][2], k


def blocked_mean(x, min_blocks=MIN_BLOCKS):
    """Mean per sample and its blocked stderr."""
    return blocked_ratio(x, None, min_blocks)

"""Workflows over several runs, as the paper's results use them (Sec. IV.A,
Sec. V.B): the initiator extrapolation I_limit -> 0 and the angularly-averaged
susceptibility from runs with small in-plane fields.

Every run is an independent ``ddqmc.Run`` stepped on the GPU; the helpers
here only combine their blocked estimates (weighted linear fits and the
angular average), so they take a run factory and can be checked on the host
with made-up estimates.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, Iterable, List, Sequence, Tuple

import numpy as np


def weighted_line(x: Sequence[float], y: Sequence[float], err: Sequence[float]) -> Tuple[float, float, float, float]:
    """Weighted least-squares line y = a + b x (weights 1/err^2): returns
    (a, sigma_a, b, sigma_b)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    w = 1.0 / np.asarray(err, dtype=float) ** 2
    S, Sx, Sy = w.sum(), (w * x).sum(), (w * y).sum()
    Sxx, Sxy = (w * x * x).sum(), (w * x * y).sum()
    D = S * Sxx - Sx * Sx
    if D <= 0:
        raise ValueError("need at least two distinct abscissae")
    a = (Sxx * Sy - Sx * Sxy) / D
    b = (S * Sxy - Sx * Sy) / D
    return a, math.sqrt(Sxx / D), b, math.sqrt(S / D)


def initiator_extrapolation(values: Dict[int, Tuple[float, float]], use: int = 3) -> Tuple[float, float]:
    """Extrapolate an observable to I_limit = 0 from its estimates at several
    initiator thresholds (Sec. IV.A, Fig. init): a weighted straight line
    through the `use` lowest thresholds, evaluated at 0.  values: {n_a:
    (estimate, blocked error)}.  Returns (value at 0, its error)."""
    keys = sorted(values)[:use]
    if len(keys) < 2:
        raise ValueError("need at least two initiator thresholds")
    a, sa, _, _ = weighted_line(keys, [values[k][0] for k in keys], [values[k][1] for k in keys])
    return a, sa


def susceptibility_tensor(mag: Callable[[int, float], Tuple[float, float, float, float]],
                          fields: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    """Linear response chi_ab = dM_a/dh_b at h = 0 (Sec. V.B): for each field
    direction b (0 = x, 1 = y) a weighted line of M_a against h through the
    fields given (h = 0 included by the caller if wanted).  mag(axis, h) ->
    (M_x, err_x, M_y, err_y).  Returns (chi, sigma_chi), 2 x 2 each."""
    chi = np.zeros((2, 2))
    err = np.zeros((2, 2))
    for b in range(2):
        est = [mag(b, h) for h in fields]
        for a in range(2):
            y = [e[2 * a] for e in est]
            # without a field M_x = M_y = 0 exactly (parity) and the blocked error is 0
            ey = [e[2 * a + 1] if (math.isfinite(e[2 * a + 1]) and e[2 * a + 1] > 0) else 1e-12 for e in est]
            _, _, slope, sslope = weighted_line(fields, y, ey)
            chi[a, b], err[a, b] = slope, sslope
    return chi, err


def angular_average(chi: np.ndarray, n: int = 720) -> float:
    """chi_av = (1/2pi) integral over theta of |chi (cos theta, sin theta)| (Sec. V.B)."""
    th = (np.arange(n) + 0.5) * (2 * np.pi / n)
    v = chi @ np.vstack([np.cos(th), np.sin(th)])
    return float(np.mean(np.hypot(v[0], v[1])))


def run_magnetisation(make_run: Callable[..., object], steps: int, axis: int, h: float,
                      n_a_values: Iterable[int] = (0,)) -> Tuple[float, float, float, float]:
    """M_x, M_y of runs at field h along `axis`, extrapolated to I_limit = 0
    over the initiator thresholds given (one threshold: that run's estimate).
    make_run(n_a=, field_h=, field_axis=) must return a ddqmc.Run."""
    per = {}
    for n_a in n_a_values:
        run = make_run(n_a=n_a, field_h=h, field_axis=axis)
        run.step(steps)
        e = run.estimates()
        run.close()
        per[n_a] = (e.mx, e.mx_err, e.my, e.my_err)
    if len(per) == 1:
        return next(iter(per.values()))
    mx = initiator_extrapolation({k: (v[0], v[1]) for k, v in per.items()})
    my = initiator_extrapolation({k: (v[2], v[3]) for k, v in per.items()})
    return mx[0], mx[1], my[0], my[1]


def trace_run(run, steps: int, every: int = 1) -> List[dict]:
    """Per-step record of a run, every `every` steps: t, shift S, trace of
    Re rho, N_w, total walkers W, occupied configurations M and the spawn
    records of the last step (the quantities of Sec. III.C's population
    control).  Returns one dict per record."""
    rows = []
    for _ in range(0, steps, every):
        run.step(every)
        st = run.state()
        est = run.raw_estimates()
        rec = run.counts()[0]
        rows.append(dict(t=int(st.t), shift=float(st.shift), trace=int(est[0]), nw=int(est[2]),
                         walkers=int(est[3]), entries=int(est[4]), spawn_records=int(rec)))
    return rows


def rows_to_csv(rows: List[dict]) -> str:
    """The records of trace_run as CSV text (header line first)."""
    if not rows:
        return ""
    keys = list(rows[0])
    return "\n".join([",".join(keys)] + [",".join(str(r[k]) for k in keys) for r in rows]) + "\n"

"""Oracle estimators, shift update, invariants and the 2x2 steady state."""
import json
import math
import os

import numpy as np
import pytest

from oracle import blocking as Bk
from oracle import exact as E
from oracle import oracle as O

C1 = dict(Lx=2, Ly=2, periodic=0, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01)


def _c1(**kw):
    p = dict(C1)
    p.update(kw)
    return O.OracleRun(p["Lx"], p["Ly"], p["periodic"], p["Jx"], p["Jy"], p["Jz"], p["gamma"],
                       p["dt"], p.get("target", 10 ** 4), n_a=p.get("n_a", 0), seed=p.get("seed", 1),
                       guide_kind=p.get("guide_kind", 0), guide_p=p.get("guide_p", 0.0))


def test_estimator_numerators_are_traces_with_matrices():
    """Integer numerators equal Re Tr(rho O) with O built from Pauli matrices."""
    rng = np.random.default_rng(3)
    run = _c1()
    N, B = run.N, run.B
    lay = O.observable_layout(N, B)
    d = 2 ** N
    entries = {}
    for _ in range(120):
        i, j = int(rng.integers(d)), int(rng.integers(d))
        entries[(i, j)] = (int(rng.integers(-50, 50)), int(rng.integers(-50, 50)))
    for i in range(d):
        entries[(i, i)] = (int(rng.integers(-50, 50)), int(rng.integers(-50, 50)))
    entries = {k: v for k, v in entries.items() if v != (0, 0)}
    keys = sorted(entries, key=lambda k: (k[1], k[0]))
    run.import_([k[0] for k in keys], [k[1] for k in keys], [entries[k][0] for k in keys],
                [entries[k][1] for k in keys])
    est = run.estimates_now()
    rho = np.zeros((d, d), dtype=complex)
    for (i, j), (re, im) in entries.items():
        rho[i, j] = re + 1j * im
    bonds = E.lattice_bonds(2, 2, 0)
    assert est[lay["tr"]] == round(np.trace(rho).real)
    assert est[lay["tr_im"]] == round(np.trace(rho).imag)
    assert est[lay["nw"]] == sum(abs(entries[(i, i)][0]) for i in range(d) if (i, i) in entries)
    assert est[lay["walkers"]] == sum(abs(a) + abs(b) for a, b in entries.values())
    assert est[lay["entries"]] == len(entries)
    for k in range(N):
        assert est[lay["z"] + k] == round(E.expect(rho, E.site_op(E.SZ, k, N)).real)
    for b, (s0, s1) in enumerate(bonds):
        for name, op in (("zz", E.SZ), ("xx", E.SX), ("yy", E.SY)):
            ref = E.expect(rho, E.site_op(op, s0, N) @ E.site_op(op, s1, N)).real
            assert est[lay[name] + b] == round(ref), (name, b)
    assert est[lay["sum_z"]] == est[lay["z"]:lay["z"] + N].sum()
    assert est[lay["sum_xx"]] == est[lay["xx"]:lay["xx"] + B].sum()
    # single-site sigma^x, sigma^y (non-zero only with entries of odd parity: the field)
    for k in range(N):
        for name, op in (("x", E.SX), ("y", E.SY)):
            ref = E.expect(rho, E.site_op(op, k, N)).real
            assert est[lay[name] + k] == round(ref), (name, k)
    assert est[lay["sum_x"]] == est[lay["x"]:lay["x"] + N].sum()
    assert est[lay["sum_y"]] == est[lay["y"]:lay["y"] + N].sum()
    assert lay["nobs"] == len(est)


def test_shift_follows_log_update():
    """S(t) = S(t-dt) + (delta/dt) log(N_w(t)/N_w(t-dt)) once the target is reached
    (Sec. III.C), S = S0 before; checked with libm's log on the recorded N_w."""
    run = _c1(target=3000)
    prev = run.state()
    Qprev = 1000
    switched = False
    for _ in range(600):
        run.step(1)
        st = run.state()
        Q = int(run.estimates_now()[2])
        if prev["variable"]:
            expect = prev["S"] + (0.05 / 0.01) * math.log(Q / Qprev)
            assert abs(st["S"] - expect) < 1e-12
        else:
            assert st["S"] == -1.0
            if Q >= 3000:
                switched = True
                assert st["variable"] == 1 and st["t_var"] == st["t"]
                assert st["t_eq"] == st["t"] + math.ceil(10 / (1.0 * 0.01))
        prev, Qprev = st, Q
    assert switched


def test_growth_phase_trace_rate():
    """Before the shift is switched on, E[Tr] grows by (1 - dt S0) per step."""
    traces = []
    for seed in range(40):
        run = _c1(target=10 ** 12, seed=seed)
        run.step(50)
        traces.append(run.estimates_now()[0])
    expect = 1000 * (1 + 0.01) ** 50
    sd = np.std(traces, ddof=1) / math.sqrt(len(traces))
    assert abs(np.mean(traces) - expect) < 4 * sd


def test_invariants_every_step():
    run = _c1(target=4000, n_a=2)
    for _ in range(300):
        run.step(1)
        k, b, r, i = run.export()
        assert np.all((r != 0) | (i != 0))
        key = b.astype(object) * (1 << 32) + k.astype(object)
        assert all(key[n] < key[n + 1] for n in range(len(key) - 1))
        pc = np.array([bin(int(x)).count("1") for x in k]) + np.array([bin(int(x)).count("1") for x in b])
        assert np.all(pc % 2 == 0)
        assert np.all(k < 16) and np.all(b < 16)


def test_dark_state_when_jx_equals_jy():
    """Jx = Jy: the all-down configuration has no off-diagonal element, so the
    walkers never leave |down..down><down..down| (and M_z = -1 exactly)."""
    run = O.OracleRun(2, 2, 0, 1.0, 1.0, 0.7, 1.0, 0.01, 5000, seed=4)
    run.step(800)
    k, b, r, i = run.export()
    assert list(k) == [0] and list(b) == [0] and i[0] == 0 and r[0] > 0
    L = E.liouvillian(2, 2, 0, 1.0, 1.0, 0.7, 1.0)
    rho, _, _ = E.ness_dense(L, 16)
    assert abs(E.observables(rho, 2, 2, 0)["mz"] + 1.0) < 1e-12


def test_single_site_relaxes_down():
    """One site, no bonds: the steady state is |down><down| (pure decay)."""
    run = O.OracleRun(1, 1, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 5000, seed=5)
    run.import_([0, 1], [0, 1], [200, 300], [0, 0])
    run.step(2000)
    k, b, r, i = run.export()
    assert list(k) == [0] and list(b) == [0]


@pytest.mark.slow
def test_ness_2x2_within_blocked_errors(golden_dir):
    """Config: 2x2 open, J = (0.9, 1, 1), gamma = 1, dt = 0.01, N_w target 10^4,
    no initiator, seed 1, 2 x 10^4 steps.  M_z within 3 blocked standard errors
    of the exact null vector; NN correlators within 4 (several comparisons)."""
    g = json.load(open(os.path.join(golden_dir, "ness_2x2_open.json")))
    run = _c1(target=10 ** 4, seed=1)
    run.step(20000)
    ser = run.series()
    assert len(ser) > 15000
    lay = O.observable_layout(4, 4)
    R, err, lvl = Bk.blocked_ratio(ser[:, lay["sum_z"]], ser[:, 0] * 4)
    assert lvl is not None and abs(R - g["mz"]) < 3 * err, (R, err, g["mz"])
    for name in ("xx", "yy", "zz"):
        R, err, _ = Bk.blocked_ratio(ser[:, lay["sum_" + name]], ser[:, 0] * 4)
        assert abs(R - np.mean(g[name])) < 4 * err, (name, R, err)
    # the shift settles at the steady-state eigenvalue 0 (Sec. III.A)
    assert abs(run.state()["S"]) < 0.2


@pytest.mark.slow
def test_ness_2x2_field_at_a_general_angle():
    """2x2 open with the in-plane field h = 0.3 at theta = 0.7 (Sec. V.B: both
    sigma^x and sigma^y in H_ext, so every field flip has a real and an
    imaginary part): M_x, M_y and M_z within 3.5 blocked errors of the exact
    null vector of the same Liouvillian (dense SVD, computed here).  N_w
    target 3000, seed 7, 1.5 x 10^4 steps."""
    h, theta = 0.3, 0.7
    L = E.liouvillian(2, 2, 0, 0.9, 1.0, 1.0, 1.0, h=h, theta=theta)
    rho, _, _ = E.ness_dense(L, 16)
    ref = {name: np.mean([E.expect(rho, E.site_op(op, k, 4)).real for k in range(4)])
           for name, op in (("x", E.SX), ("y", E.SY), ("z", E.SZ))}
    run = O.OracleRun(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 3000, seed=7, field_h=h, field_axis=2,
                      field_theta=theta)
    run.step(15000)
    ser = run.series()
    assert len(ser) > 12000
    lay = O.observable_layout(4, 4)
    for name in ("x", "y", "z"):
        R, err, _ = Bk.blocked_ratio(ser[:, lay["sum_" + name]], ser[:, 0] * 4)
        assert abs(R - ref[name]) < 3.5 * err, (name, R, err, ref[name])
    # both in-plane components are sizeable at this angle
    assert abs(ref["x"]) > 0.05 and abs(ref["y"]) > 0.05

"""Host-side combination of runs: weighted line fits (against numpy's weighted
polyfit), the initiator extrapolation, the susceptibility tensor from
magnetisations and its angular average (against the complete elliptic
integral for a diagonal tensor)."""
import math

import numpy as np
import pytest

from paper_1802_05931_gb300 import workflows as WF


def test_weighted_line_matches_polyfit():
    rng = np.random.default_rng(1)
    x = np.array([0.0, 1.0, 2.5, 4.0, 7.0])
    err = rng.uniform(0.1, 0.5, size=5)
    y = 0.3 - 1.7 * x + rng.normal(0, err)
    a, sa, b, sb = WF.weighted_line(x, y, err)
    (pb, pa), cov = np.polyfit(x, y, 1, w=1 / err, cov="unscaled")
    assert a == pytest.approx(pa, rel=1e-12) and b == pytest.approx(pb, rel=1e-12)
    assert sa == pytest.approx(math.sqrt(cov[1, 1]), rel=1e-10)
    assert sb == pytest.approx(math.sqrt(cov[0, 0]), rel=1e-10)


def test_initiator_extrapolation_uses_the_lowest_thresholds():
    vals = {3: (0.5 + 0.01 * 3, 0.01), 6: (0.5 + 0.01 * 6, 0.01), 10: (0.5 + 0.01 * 10, 0.02),
            40: (9.0, 0.01)}                      # far outlier, not among the three lowest
    v, e = WF.initiator_extrapolation(vals)
    assert v == pytest.approx(0.5, abs=1e-12) and e > 0


def test_susceptibility_tensor_from_linear_magnetisation():
    chi = np.array([[0.2, -3.8], [3.4, 2.7]])

    def mag(axis, h):
        m = chi[:, axis] * h
        return m[0], 0.01, m[1], 0.01
    got, err = WF.susceptibility_tensor(mag, [0.0, 0.02, 0.04])
    assert np.allclose(got, chi, atol=1e-12) and np.all(err > 0)


def test_angular_average_of_diagonal_tensor_is_an_elliptic_integral():
    scipy_special = pytest.importorskip("scipy.special")
    a, b = 3.0, 1.2
    ref = (2 / math.pi) * a * scipy_special.ellipe(1 - (b / a) ** 2)
    assert WF.angular_average(np.diag([a, b])) == pytest.approx(ref, rel=1e-6)
    assert WF.angular_average(2.5 * np.eye(2)) == pytest.approx(2.5, rel=1e-12)


def test_trace_run_records_every_interval():
    import types

    class Fake:
        def __init__(self):
            self.t = 0

        def step(self, n):
            self.t += n

        def state(self):
            return types.SimpleNamespace(t=self.t, shift=0.5 * self.t)

        def raw_estimates(self):
            return [self.t, 0, 2 * self.t, 3 * self.t, 4 * self.t]

        def counts(self):
            return (5 * self.t, 0, 0)

    rows = WF.trace_run(Fake(), 10, every=5)
    assert [r["t"] for r in rows] == [5, 10]
    assert rows[1] == dict(t=10, shift=5.0, trace=10, nw=20, walkers=30, entries=40, spawn_records=50)
    csv = WF.rows_to_csv(rows).splitlines()
    assert csv[0] == "t,shift,trace,nw,walkers,entries,spawn_records" and csv[2].startswith("10,5.0,")


def test_angular_average_from_the_tensor_equals_the_direct_average():
    """chi_av of Sec. V.B read as the angle average of the response to a
    field at each angle (reading 22 takes it from the 2 x 2 tensor of the x
    and y responses).  On the exact 2x2 steady state (dense null vectors of
    the Liouvillian with the field at each angle) both agree to O(h)."""
    from oracle import exact as E
    h = 1e-3

    def mag(theta):
        L = E.liouvillian(2, 2, 0, 0.9, 1.0, 1.0, 1.0, h=h, theta=theta)
        rho, _, _ = E.ness_dense(L, 16)
        return np.array([np.mean([E.expect(rho, E.site_op(op, k, 4)).real for k in range(4)])
                          for op in (E.SX, E.SY)])

    chi = np.column_stack([mag(0.0) / h, mag(np.pi / 2) / h])
    n = 48
    thetas = (np.arange(n) + 0.5) * (2 * np.pi / n)
    direct = [np.hypot(*mag(t)) / h for t in thetas]
    # the tensor predicts the response at every angle (linear response)
    for t, d in zip(thetas[::8], direct[::8]):
        pred = chi @ np.array([np.cos(t), np.sin(t)])
        assert np.hypot(*pred) == pytest.approx(d, rel=5e-3, abs=1e-6)
    assert WF.angular_average(chi, n=n) == pytest.approx(float(np.mean(direct)), rel=5e-3)
    assert WF.angular_average(chi) > 0.05          # a finite in-plane susceptibility

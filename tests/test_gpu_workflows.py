"""The susceptibility workflow of Sec. V.B on the GPU: 2x2 open lattice, runs
with small in-plane fields along x and along y, linear response tensor from
weighted fits of M_x, M_y against h, compared with the same fits through the
exact steady-state magnetisations of the Liouvillian (within 4 errors)."""
import numpy as np
import pytest

from oracle import exact as E
from tests import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = [0.0, 0.02, 0.04]


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc, workflows
    return ddqmc, workflows


def _exact_mag(axis, h):
    L = E.liouvillian(2, 2, 0, 0.9, 1.0, 1.0, 1.0, h=h, theta=axis * np.pi / 2)
    rho, _, _ = E.ness_dense(L, 16)
    ob = E.observables(rho, 2, 2, 0)
    return np.mean(ob["x"]), 1.0, np.mean(ob["y"]), 1.0


def test_susceptibility_of_2x2_against_exact(mods):
    ddqmc, WF = mods
    args, kw = W.run_kwargs(W.C1)

    def make_run(n_a, field_h, field_axis):
        k = dict(kw, n_a=n_a, field_h=field_h, field_axis=field_axis)
        return ddqmc.Run(*args, **k)

    def mag(axis, h):
        return WF.run_magnetisation(make_run, W.C1["steps"], axis, h)
    chi, err = WF.susceptibility_tensor(mag, FIELDS)
    chi_x, _ = WF.susceptibility_tensor(_exact_mag, FIELDS)
    assert np.all(np.abs(chi - chi_x) < 4 * err + 1e-9), (chi, chi_x, err)
    assert abs(WF.angular_average(chi) - WF.angular_average(chi_x)) < 0.15 * WF.angular_average(chi_x)

"""Pins of the sparse steady-state solver (oracle/exact.py ness_sparse).

The 3x3 steady states that the GPU observables are compared with (Sec. V.A)
come from ness_sparse: Runge-Kutta propagation restricted to the
configurations reachable from the all-down state.  These tests pin it to
things other than itself:

* on lattices small enough for a dense SVD null vector (2x2 open, rings of
  three and five sites with periodic bonds) the sparse solution equals the
  dense one, with two coupling sets;
* the residual is taken with the FULL Liouvillian, not the sector, so a
  sector that leaves out configurations the dynamics reach shows up as a
  residual;
* the stored 3x3 goldens are recomputed here and must reproduce their stored
  observables, be unit-trace, Hermitian and positive semidefinite, and have a
  full-Liouvillian residual below 1e-10;
* for Jx = Jy (the XXZ case) the all-down state is dark: the Hamiltonian
  conserves the magnetisation and annihilates nothing out of |down..down>, so
  the steady state is |down..down><down..down| with M_z = -1 exactly.
"""
import json
import os

import numpy as np
import pytest

from oracle import exact as E

COUPLINGS = [(0.9, 1.0, 1.0), (0.225, 0.335, 0.25)]
SMALL = [(2, 2, 0), (3, 1, 1), (5, 1, 1)]


def _full_residual(L, rho):
    v = rho.reshape(-1, order="F")
    return np.linalg.norm(L @ v) / np.linalg.norm(v)


def _compare(a, b, tol):
    for key in ("z", "x", "y", "xx", "yy", "zz"):
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=tol, err_msg=key)
    assert abs(a["mz"] - b["mz"]) < tol


@pytest.mark.parametrize("lat", SMALL)
@pytest.mark.parametrize("J", COUPLINGS)
def test_sparse_equals_dense_null_vector(lat, J):
    Lx, Ly, per = lat
    N = Lx * Ly
    d = 2 ** N
    L = E.liouvillian(Lx, Ly, per, *J, 1.0)
    rho_d, s_min, s_next = E.ness_dense(L, d)
    assert s_min < 1e-10 < s_next          # a unique steady state
    rho_s, resid = E.ness_sparse(L, d)
    assert resid < 1e-10
    assert _full_residual(L, rho_s) < 1e-10
    assert abs(np.trace(rho_s) - 1.0) < 1e-12
    np.testing.assert_allclose(rho_s, rho_d, rtol=0, atol=1e-9)
    _compare(E.observables(rho_s, Lx, Ly, per), E.observables(rho_d, Lx, Ly, per), 1e-9)


def test_sector_keeps_only_even_parity_and_starts_at_all_down():
    d = 8
    keep = E.sector_indices(d)
    assert keep[0] == 0                    # vec index 0 is |0><0|, the initial state
    assert len(keep) == d * d // 2
    for v in keep:
        i, j = v % d, v // d
        assert (bin(i).count("1") + bin(j).count("1")) % 2 == 0


@pytest.mark.parametrize("lat", [(2, 2, 0), (3, 3, 1)])
def test_xxz_dark_state(lat):
    Lx, Ly, per = lat
    d = 2 ** (Lx * Ly)
    L = E.liouvillian(Lx, Ly, per, 0.7, 0.7, 1.3, 1.0)
    rho, resid = E.ness_sparse(L, d)
    assert resid < 1e-12
    assert abs(rho[0, 0] - 1.0) < 1e-12
    assert np.count_nonzero(np.abs(rho) > 1e-12) == 1
    assert abs(E.observables(rho, Lx, Ly, per)["mz"] + 1.0) < 1e-12


@pytest.fixture(scope="module")
def stored_3x3(golden_dir):
    out = []
    for name in ("ness_3x3_periodic.json", "ness_3x3_periodic_weak.json"):
        with open(os.path.join(golden_dir, name)) as f:
            g = json.load(f)
        Lx, Ly, per = g["lattice"]
        L = E.liouvillian(Lx, Ly, per, g["Jx"], g["Jy"], g["Jz"], g["gamma"])
        rho, resid = E.ness_sparse(L, 2 ** (Lx * Ly))
        out.append((name, g, L, rho, resid))
    return out


def test_stored_3x3_goldens_are_steady_states(stored_3x3):
    for name, g, L, rho, resid in stored_3x3:
        Lx, Ly, per = g["lattice"]
        assert _full_residual(L, rho) < 1e-10, name
        assert abs(np.trace(rho) - 1.0) < 1e-12, name
        assert np.max(np.abs(rho - rho.conj().T)) < 1e-10, name
        assert np.linalg.eigvalsh(rho).min() > -1e-10, name
        ob = E.observables(rho, Lx, Ly, per)
        _compare(ob, {k: np.asarray(g[k]) if k != "mz" else g["mz"]
                      for k in ("z", "x", "y", "xx", "yy", "zz", "mz")}, 1e-9)
        # translation invariance of the periodic lattice: every site alike
        assert np.ptp(ob["z"]) < 1e-9, name

"""The oracle's move generator against the Kronecker form of the shifted
Liouvillian (Nagy & Savona, Sec. III.C), built from Pauli matrices."""
import itertools

import numpy as np
import pytest

from oracle import exact as E
from oracle import oracle as O

LATTICES = [(2, 2, 0), (3, 1, 1), (1, 3, 0), (2, 3, 0), (3, 1, 0)]


@pytest.mark.parametrize("Lx,Ly,per", LATTICES)
def test_bonds_match(Lx, Ly, per):
    r = O.OracleRun(Lx, Ly, per, 0.9, 1.0, 1.0, 1.0, 0.01, 100)
    assert r.bonds() == E.lattice_bonds(Lx, Ly, per)


# (h, axis, theta): none, along x, along y, and at general angles (axis 2),
# where every site flip has a real and an imaginary part
FIELDS = [(0.0, 0, 0.0), (0.37, 0, 0.0), (-0.55, 1, 0.0), (0.45, 2, 0.7), (-0.3, 2, 2.3)]


def _theta(axis, theta):
    return theta if axis == 2 else axis * np.pi / 2


@pytest.mark.parametrize("Lx,Ly,per", LATTICES)
@pytest.mark.parametrize("J", [(0.9, 1.0, 1.0), (0.3, -1.2, 0.7), (1.1, 1.1, -0.4)])
@pytest.mark.parametrize("h,axis,theta", FIELDS)
def test_every_element_matches_kronecker(Lx, Ly, per, J, h, axis, theta):
    Jx, Jy, Jz = J
    gamma, S = 0.7, 0.37
    r = O.OracleRun(Lx, Ly, per, Jx, Jy, Jz, gamma, 0.01, 100, shift0=S, field_h=h, field_axis=axis,
                    field_theta=theta)
    d = 2 ** (Lx * Ly)
    L = E.liouvillian(Lx, Ly, per, Jx, Jy, Jz, gamma, S=S, h=h, theta=_theta(axis, theta)).toarray()
    rebuilt = np.zeros_like(L)
    for i, j in itertools.product(range(d), range(d)):
        ck, cb, kind, A, rate = r.moves(i, j)
        assert len(A) == 2 * r.B + r.N + ((4 if axis == 2 else 2) * r.N if h else 0)
        # every move has a purely real or a purely imaginary element
        assert np.all((A.real == 0) | (A.imag == 0))
        p = E.vec_index(i, j, d)
        for a, b, amp in zip(ck, cb, A):
            if amp != 0:
                rebuilt[E.vec_index(int(a), int(b), d), p] += amp
        rebuilt[p, p] += r.diag(i, j)
    assert np.abs(L - rebuilt).max() < 1e-13


def _weight(i, j, kind, p, r_site, N):
    """Importance weight of configuration (i, j) from its definition (Sec. IV.B)."""
    if i == j:
        return 1.0
    if kind == 1:
        return float(np.exp(-p))
    w = 1.0
    for k in range(N):
        if ((i >> k) & 1) != ((j >> k) & 1):
            w *= r_site[k]
    return w


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("h,axis,theta", FIELDS)
def test_rates_are_truncated_scaled_elements(kind, h, axis, theta):
    """Each fixed-point rate is |A| dt w(child)/w(parent) * 2^32 truncated (to within
    the rounding of the product order)."""
    Lx, Ly, per = 2, 2, 0
    dt, p = 0.05, 1.3
    r_site = [0.5, 0.7, 0.9, 0.6]
    r = O.OracleRun(Lx, Ly, per, 0.9, 1.0, 1.0, 1.0, dt, 100, guide_kind=kind, guide_p=p,
                    site_ratio=r_site if kind == 2 else None, field_h=h, field_axis=axis, field_theta=theta)
    d = 16
    for i, j in itertools.product(range(d), range(d)):
        ck, cb, _, A, rate = r.moves(i, j)
        for a, b, amp, q in zip(ck, cb, A, rate):
            ratio = 1.0
            if kind:
                ratio = _weight(int(a), int(b), kind, p, r_site, 4) / _weight(i, j, kind, p, r_site, 4)
            expect = abs(amp) * dt * ratio * 2.0 ** 32
            assert abs(int(q) - expect) <= 1.0 + 1e-9 * expect, (i, j, a, b, q, expect)


@pytest.mark.parametrize("h,axis,theta", [(0.4, 0, 0.0), (-0.35, 1, np.pi / 2)])
def test_general_angle_reduces_to_the_axes(h, axis, theta):
    """At theta = 0 and theta = pi/2 the general-angle moves carry the x-axis
    (resp. y-axis) elements and rates, with zero-rate moves in between that
    leave every cumulative threshold unchanged: the runs are bit-identical."""
    a = O.OracleRun(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 5000, seed=9, n_a=2, field_h=h, field_axis=axis)
    b = O.OracleRun(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 5000, seed=9, n_a=2, field_h=h, field_axis=2,
                    field_theta=theta)
    for t in range(150):
        a.step(1)
        b.step(1)
        for x, y in zip(a.export(), b.export()):
            assert np.array_equal(x, y), t
        assert np.array_equal(a.estimates_now(), b.estimates_now()), t

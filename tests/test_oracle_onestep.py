"""One oracle step is an unbiased sample of the Euler step of the shifted
Liouvillian: E[rho(t+dt) | rho(t)] = (1 + dt L~) rho(t) (Sec. III.A, Euler
equation), element by element, with and without importance sampling
(Sec. IV.B, where the off-diagonal elements become w_child L~ / w_parent).
The trace therefore scales by exactly (1 - dt S) in expectation."""
import numpy as np
import pytest

from oracle import exact as E
from oracle import oracle as O

# a 2x2 state with diagonal and off-diagonal entries, real and imaginary parts
STATE = [  # (ket, bra, re, im)
    (0, 0, 60, 0), (3, 3, 25, -7), (3, 0, 9, 8), (5, 6, -6, 3), (15, 12, 4, -4), (0, 9, 0, 5),
]


def _dense(state, d):
    rho = np.zeros((d, d), dtype=complex)
    for i, j, re, im in state:
        rho[i, j] = re + 1j * im
    return rho


def _weights(d, kind, p, r_site, N):
    w = np.ones((d, d))
    for i in range(d):
        for j in range(d):
            if i == j:
                continue
            if kind == 1:
                w[i, j] = np.exp(-p)
            elif kind == 2:
                for k in range(N):
                    if ((i >> k) & 1) != ((j >> k) & 1):
                        w[i, j] *= r_site[k]
    return w


def _sorted(state):
    return sorted(state, key=lambda e: (e[1], e[0]))


CASES = [
    # dt, S, guide kind, p, site ratios, field h, field axis, samples
    (0.05, 0.3, 0, 0.0, None, 0.0, 0, 2500),
    (0.2, -6.0, 1, 1.5, None, 0.0, 0, 2500),     # n_att > 1 attempts and |p_death| > 1
    (0.1, 0.5, 2, 0.0, [0.5, 0.7, 0.9, 0.6], 0.0, 0, 2500),
    (0.1, 0.5, 0, 0.0, None, 0.8, 0, 2500),      # in-plane field along x
    (0.1, 0.5, 2, 0.0, [0.5, 0.7, 0.9, 0.6], -0.6, 1, 2500),   # along y, site-product guide
    (0.1, 0.2, 1, 1.2, None, 0.5, 1, 2500),
    (0.1, 0.5, 0, 0.0, None, 0.7, 2, 2500),      # general angle 0.7: real and imaginary parts
    (0.1, 0.5, 2, 0.0, [0.5, 0.7, 0.9, 0.6], -0.6, 2, 2500),
]
THETA = 0.7                                     # the angle of the axis-2 cases


@pytest.mark.parametrize("dt,S,kind,p,r_site,h,axis,ns", CASES)
def test_one_step_is_unbiased(dt, S, kind, p, r_site, h, axis, ns):
    Jx, Jy, Jz, gamma = 0.9, 1.0, 1.3, 1.0
    d = 16
    run = O.OracleRun(2, 2, 0, Jx, Jy, Jz, gamma, dt, 10 ** 15, n_a=0, guide_kind=kind,
                      guide_p=p, site_ratio=r_site, seed=11, shift0=S, field_h=h, field_axis=axis,
                      field_theta=THETA)
    st = _sorted(STATE)
    ket = [e[0] for e in st]; bra = [e[1] for e in st]; re = [e[2] for e in st]; im = [e[3] for e in st]
    acc = np.zeros((d, d), dtype=complex)
    acc2r = np.zeros((d, d))
    acc2i = np.zeros((d, d))
    for s in range(ns):
        run.import_(ket, bra, re, im)
        run.set_state(s, S, 0, 1, -1, -1)          # t = s selects independent draws
        run.step(1)
        k2, b2, r2, i2 = run.export()
        rho = np.zeros((d, d), dtype=complex)
        rho[k2.astype(int), b2.astype(int)] = r2 + 1j * i2
        acc += rho
        acc2r += rho.real ** 2
        acc2i += rho.imag ** 2
    mean = acc / ns
    L = E.liouvillian(2, 2, 0, Jx, Jy, Jz, gamma, S=S, h=h,
                      theta=THETA if axis == 2 else axis * np.pi / 2).toarray()
    if kind:
        w = _weights(d, kind, p, r_site, 4).reshape(-1, order="F")
        off = ~np.eye(d * d, dtype=bool)
        L = np.where(off, L * w[:, None] / w[None, :], L)
    rho0 = _dense(STATE, d).reshape(-1, order="F")
    expect = (rho0 + dt * (L @ rho0)).reshape((d, d), order="F")
    var_r = np.maximum(acc2r / ns - mean.real ** 2, 1e-12)
    var_i = np.maximum(acc2i / ns - mean.imag ** 2, 1e-12)
    zr = (mean.real - expect.real) / np.sqrt(var_r / ns)
    zi = (mean.imag - expect.imag) / np.sqrt(var_i / ns)
    # elements never reached must be exactly zero in every sample
    never = (acc2r == 0) & (acc2i == 0)
    assert np.all(np.abs(expect[never]) < 1e-12)
    assert np.abs(zr[~never]).max() < 4.5 and np.abs(zi[~never]).max() < 4.5, (zr.max(), zi.max())
    # trace: E[Tr rho(t+dt)] = (1 - dt S) Tr rho(t)
    tr = np.trace(mean).real
    tr_expect = (1 - dt * S) * np.trace(_dense(STATE, d)).real
    tr_sd = np.sqrt(np.sum(np.diag(var_r)) / ns)
    assert abs(tr - tr_expect) < 4.5 * tr_sd + 1e-9

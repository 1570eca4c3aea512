"""Exact Liouvillian and steady state -- TEST INFRASTRUCTURE ONLY.

The exact references the oracle is pinned against (Nagy & Savona,
arXiv:1802.05931):

* the vectorised shifted Liouvillian in its Kronecker form (Sec. III.C),
  L~ = -i(1 (x) H - H^T (x) 1) - S 1 (x) 1
       + sum_k gamma/2 (2 F_k^* (x) F_k - 1 (x) F_k^dag F_k - F_k^T F_k^* (x) 1),
  with column-stacking vec(rho)[i + d*j] = rho_ij, built from explicit Pauli
  matrices and Kronecker products (no element rules);
* the XYZ Hamiltonian on nearest-neighbour bonds and sigma^- decay on every
  site (Sec. V);
* the non-equilibrium steady state, the null vector of L~ at S = 0 with unit
  trace, which is what the paper compares DDQMC against for 2x2 and 3x3
  lattices (Sec. V.A);
* observables as Tr(rho O) with O built from matrices (Sec. III.A, Sec. V.A).

Only the tests and the golden-file script use this module.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# single-site matrices in the basis (|down>, |up>): index 0 = down (bit 0), 1 = up (bit 1)
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, 1j], [-1j, 0]], dtype=complex)   # <down|sy|up> = i, <up|sy|down> = -i
SZ = np.array([[-1, 0], [0, 1]], dtype=complex)
SM = np.array([[0, 1], [0, 0]], dtype=complex)      # sigma^- = |down><up|
I2 = np.eye(2, dtype=complex)


def lattice_bonds(Lx, Ly, periodic):
    """Nearest-neighbour bonds, site k = x + Lx*y; for each site in (y, x) order
    the bond to the right, then the bond below (wrapping when periodic)."""
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            a = x + Lx * y
            if Lx > 1 and (x + 1 < Lx or periodic):
                bonds.append((a, (x + 1) % Lx + Lx * y))
            if Ly > 1 and (y + 1 < Ly or periodic):
                bonds.append((a, x + Lx * ((y + 1) % Ly)))
    return bonds


def site_op(op, k, N):
    """op acting on site k of N (basis index = sum_k bit_k 2^k)."""
    left = sp.identity(2 ** (N - 1 - k), dtype=complex, format="csr")
    right = sp.identity(2 ** k, dtype=complex, format="csr")
    return sp.kron(sp.kron(left, sp.csr_matrix(op)), right, format="csr")


def hamiltonian(N, bonds, Jx, Jy, Jz, h=0.0, theta=0.0):
    """XYZ bonds plus the in-plane field h sum_k (cos theta sx_k + sin theta sy_k) (Sec. V.B)."""
    d = 2 ** N
    H = sp.csr_matrix((d, d), dtype=complex)
    for a, b in bonds:
        H = H + Jx * (site_op(SX, a, N) @ site_op(SX, b, N))
        H = H + Jy * (site_op(SY, a, N) @ site_op(SY, b, N))
        H = H + Jz * (site_op(SZ, a, N) @ site_op(SZ, b, N))
    if h != 0.0:
        F = np.cos(theta) * SX + np.sin(theta) * SY
        for k in range(N):
            H = H + h * site_op(F, k, N)
    return H.tocsr()


def liouvillian(Lx, Ly, periodic, Jx, Jy, Jz, gamma, S=0.0, h=0.0, theta=0.0):
    """Shifted vectorised Liouvillian (d^2 x d^2, sparse), Kronecker form."""
    N = Lx * Ly
    d = 2 ** N
    bonds = lattice_bonds(Lx, Ly, periodic)
    H = hamiltonian(N, bonds, Jx, Jy, Jz, h, theta)
    Id = sp.identity(d, dtype=complex, format="csr")
    L = -1j * (sp.kron(Id, H) - sp.kron(H.T, Id)) - S * sp.identity(d * d, dtype=complex)
    for k in range(N):
        F = site_op(SM, k, N)
        FdF = (F.conj().T @ F).tocsr()
        L = L + (gamma / 2.0) * (2.0 * sp.kron(F.conj(), F) - sp.kron(Id, FdF)
                                 - sp.kron((F.T @ F.conj()).tocsr(), Id))
    return L.tocsr()


def vec_index(i, j, d):
    return i + d * j


def ness_dense(L, d):
    """Null vector of a dense L~ (S = 0) by SVD, normalised to unit trace."""
    Ld = L.toarray() if sp.issparse(L) else np.asarray(L)
    _, s, vh = np.linalg.svd(Ld)
    v = vh[-1].conj()
    rho = v.reshape((d, d), order="F")
    rho = rho / np.trace(rho)
    rho = 0.5 * (rho + rho.conj().T)
    return rho, s[-1], s[-2]


def sector_indices(d):
    """vec indices of the configurations reached from |down..down><down..down|:
    every move flips an even number of spins across ket and bra together, so
    popcount(i) + popcount(j) stays even."""
    idx = np.arange(d * d)
    i = idx % d
    j = idx // d
    pc = np.array([bin(x).count("1") for x in range(d)])
    return np.nonzero((pc[i] + pc[j]) % 2 == 0)[0]


def ness_sparse(L, d, tol=1e-11, dt=None, max_time=2000.0, check_every=50):
    """Null vector of a sparse L~ (S = 0) with unit trace, in the sector
    reached from the all-down state.

    Classical fourth-order Runge-Kutta propagation of d rho/dt = L~ rho from
    |down..down><down..down|.  Its step map is a polynomial p(dt L~) with
    p(0) = 1, so the null vector is an exact fixed point and every other mode
    (Re lambda < 0) decays when dt lambda is inside the stability region;
    propagation stops when ||L~ rho|| / ||rho|| < tol.

    Step: the eigenvalues of a Lindblad generator lie in the closed left
    half-plane, every eigenvalue is bounded by the largest absolute row sum
    (Gershgorin), and the left half-disc of radius 2.5 lies inside the
    classical RK4 stability region, so dt = 2.5 / max_row_sum |L~| is stable
    for every mode.  (An estimate of the spectral radius by power iteration
    is not a bound: on a three-site ring it came out at half the true radius
    and the propagation diverged.)"""
    keep = sector_indices(d)
    Ls = L[keep][:, keep].tocsr()
    n = len(keep)
    if dt is None:
        dt = 2.5 / float(abs(Ls).sum(axis=1).max())
    x = np.zeros(n, dtype=complex)
    x[0] = 1.0                          # vec index 0 is |0><0| = all down
    t = 0.0
    step = 0
    resid = np.inf
    while t < max_time:
        k1 = Ls @ x
        if step % check_every == 0:
            resid = np.linalg.norm(k1) / np.linalg.norm(x)
            if resid < tol:
                break
        k2 = Ls @ (x + (0.5 * dt) * k1)
        k3 = Ls @ (x + (0.5 * dt) * k2)
        k4 = Ls @ (x + dt * k3)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        t += dt
        step += 1
    full = np.zeros(d * d, dtype=complex)
    full[keep] = x
    rho = full.reshape((d, d), order="F")
    rho = rho / np.trace(rho)
    resid = np.linalg.norm(L @ rho.reshape(-1, order="F")) / np.linalg.norm(rho)
    rho = 0.5 * (rho + rho.conj().T)
    return rho, resid


def expect(rho, O):
    """Tr(rho O) = sum_ij rho_ij O_ji."""
    if sp.issparse(O):
        O = O.tocoo()
        return complex(np.sum(rho[O.col, O.row] * O.data))
    return complex(np.sum(rho * np.asarray(O).T))


def observables(rho, Lx, Ly, periodic):
    """Steady-state observables from matrices: per-site sigma^{x,y,z}, M_z
    (Sec. V.A) and nearest-neighbour xx, yy, zz per bond."""
    N = Lx * Ly
    bonds = lattice_bonds(Lx, Ly, periodic)
    tr = np.trace(rho)
    out = {"trace": complex(tr)}
    for name, op in (("x", SX), ("y", SY), ("z", SZ)):
        out[name] = np.array([expect(rho, site_op(op, k, N)).real / tr.real for k in range(N)])
    out["mz"] = float(np.mean(out["z"]))
    for name, op in (("xx", SX), ("yy", SY), ("zz", SZ)):
        out[name] = np.array([expect(rho, site_op(op, a, N) @ site_op(op, b, N)).real / tr.real
                              for a, b in bonds])
    return out

"""Write the stored exact values the tests compare against.

Calls only ``oracle/exact.py`` (Kronecker Liouvillian and its null vector),
never the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py

Outputs (JSON, one file per lattice):
  ness_2x2_open.json            dense SVD null vector, 256 x 256 Liouvillian
  ness_3x3_periodic.json        Runge-Kutta fixed point, 262144-dim Liouvillian
  ness_3x3_periodic_weak.json   same, couplings (0.225, 0.335, 0.25)
  ness_2x2_open_field_x.json    2x2 open with the in-plane field h = 0.3 along x
  ness_2x2_open_field_y.json    the same along y (theta = pi/2), Sec. V.B
The 2x2 and first 3x3 use Jx = 0.9, Jy = 1.0, Jz = 1.0, the other 3x3 the
couplings of the paper's 3x3 figure (Sec. V.A) as Pauli couplings; all have
gamma = 1, Pauli matrices in H and sigma^- decay on every site (Nagy &
Savona, Sec. V).  ``python tests/golden/make_golden.py field`` writes only
the two field files.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402


def dump(name, Lx, Ly, periodic, rho, resid, method, J=(0.9, 1.0, 1.0), h=0.0, theta=0.0):
    ob = exact.observables(rho, Lx, Ly, periodic)
    rec = dict(lattice=[Lx, Ly, periodic], Jx=J[0], Jy=J[1], Jz=J[2], gamma=1.0, h=h, theta=theta,
               method=method, residual=float(resid), mz=ob["mz"],
               z=ob["z"].tolist(), x=ob["x"].tolist(), y=ob["y"].tolist(),
               xx=ob["xx"].tolist(), yy=ob["yy"].tolist(), zz=ob["zz"].tolist(),
               bonds=exact.lattice_bonds(Lx, Ly, periodic))
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, "mz", ob["mz"], "residual", resid)


def field_files():
    for axis, name in ((0, "ness_2x2_open_field_x.json"), (1, "ness_2x2_open_field_y.json")):
        theta = axis * np.pi / 2
        L = exact.liouvillian(2, 2, 0, 0.9, 1.0, 1.0, 1.0, h=0.3, theta=theta)
        rho, s_min, _ = exact.ness_dense(L, 16)
        resid = np.linalg.norm(L @ rho.reshape(-1, order="F"))
        dump(name, 2, 2, 0, rho, resid, "dense SVD null vector", h=0.3, theta=theta)


def main():
    field_files()
    L = exact.liouvillian(2, 2, 0, 0.9, 1.0, 1.0, 1.0)
    rho, s_min, _ = exact.ness_dense(L, 16)
    resid = np.linalg.norm(L @ rho.reshape(-1, order="F"))
    dump("ness_2x2_open.json", 2, 2, 0, rho, resid, "dense SVD null vector")
    L = exact.liouvillian(3, 3, 1, 0.9, 1.0, 1.0, 1.0)
    rho, resid = exact.ness_sparse(L, 512)
    dump("ness_3x3_periodic.json", 3, 3, 1, rho, resid, "RK4 fixed point, sector popcount(i)+popcount(j) even")
    # the couplings of the paper's 3x3 figure (Jx, Jy, Jz)/gamma = (0.225, 0.335, 0.25), taken as Pauli couplings
    J = (0.225, 0.335, 0.25)
    L = exact.liouvillian(3, 3, 1, J[0], J[1], J[2], 1.0)
    rho, resid = exact.ness_sparse(L, 512)
    dump("ness_3x3_periodic_weak.json", 3, 3, 1, rho, resid, "RK4 fixed point, sector popcount(i)+popcount(j) even", J)


if __name__ == "__main__":
    if sys.argv[1:] == ["field"]:
        field_files()
    else:
        main()

"""Seeded synthetic workloads shared by the tests and the benchmark.

Parameter sets only: no arithmetic of the method lives here.  They follow the
paper's workloads (2D XYZ lattices with sigma^- decay, Sec. V; initiator
threshold, Sec. IV.A; importance sampling, Sec. IV.B), with the couplings
Jx = 0.9, Jy = Jz = 1, gamma = 1.
"""

C1 = dict(Lx=2, Ly=2, periodic=0, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=10 ** 4,
          n_a=0, seed=1, steps=20000)
C2 = dict(Lx=3, Ly=3, periodic=1, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=10 ** 6,
          n_a=3, seed=2, steps=50000)
# 3x3 periodic with the couplings of the paper's 3x3 figure, (0.225, 0.335, 0.25),
# taken as Pauli couplings: a regime where the walker population stays near
# the diagonal target, used for the comparison with the exact steady state
C2W = dict(Lx=3, Ly=3, periodic=1, Jx=0.225, Jy=0.335, Jz=0.25, gamma=1.0, dt=0.005, target=10 ** 4,
           n_a=0, seed=2, steps=40000)
# 4x4 periodic, 10^8 walkers in total (control on the total population), n_a = 3,
# site-product guide with every site ratio exp(-1.5) (the paper's uniform
# weight per flipped site, through the site-product code path).
C3 = dict(Lx=4, Ly=4, periodic=1, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=10 ** 8,
          n_a=3, seed=3, steps=10000, control=1, guide_kind=2, guide_p=1.5)


def run_kwargs(cfg, **over):
    """Keyword arguments of ddqmc.Run / OracleRun for a config dict."""
    import math
    c = dict(cfg)
    c.update(over)
    kw = dict(n_a=c["n_a"], seed=c["seed"], control=c.get("control", 0))
    gk = c.get("guide_kind", 0)
    if gk:
        kw["guide_kind"] = gk
        kw["guide_p"] = c.get("guide_p", 0.0)
        if gk == 2:
            kw["site_ratio"] = [math.exp(-c.get("guide_p", 0.0))] * (c["Lx"] * c["Ly"])
    for k in ("n0", "shift0", "damping", "t_eq", "field_h", "field_axis", "field_theta"):
        if k in c:
            kw[k] = c[k]
    args = (c["Lx"], c["Ly"], c["periodic"], c["Jx"], c["Jy"], c["Jz"], c["gamma"], c["dt"], c["target"])
    return args, kw

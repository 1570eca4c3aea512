"""In-plane field at a general angle (Sec. V.B, H_ext = h sum_k (cos t sigma^x_k
+ sin t sigma^y_k)): each site flip is two moves, the x part (the other
walker type) and the y part (the same type).  The GPU path against the oracle,
element by element, on both spawn paths, with single runs and in a batch."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as d
    return d


def _same(gpu, cpu, where):
    g = gpu.export()
    c = cpu.export()
    assert len(g[0]) == len(c[0]), (where, len(g[0]), len(c[0]))
    for name, a, b in zip(("ket", "bra", "re", "im"), g, c):
        assert np.array_equal(a, b), (where, name)
    assert np.array_equal(gpu.raw_estimates(), cpu.estimates_now()), where


ANGLES = [
    # (base config, overrides): every quadrant of the angle, both signs of h
    ("C1", dict(field_h=0.3, field_theta=0.7)),
    ("C1", dict(field_h=-0.4, field_theta=2.3, guide_kind=1, guide_p=1.5, dt=0.02, control=1, target=5000)),
    ("C2", dict(field_h=0.25, field_theta=-1.1, guide_kind=2, guide_p=0.7, n_a=2, dt=0.01, control=1,
                target=20000)),
    ("C3", dict(field_h=0.1, field_theta=4.0, target=30000)),
]


@pytest.mark.parametrize("base,over", ANGLES)
def test_angle_bitexact(ddqmc, base, over):
    """Uniform tables: the lane-per-walker path (and the warp-cooperative one
    for the configurations above the heavy threshold)."""
    over = dict(over, field_axis=2)
    args, kw = W.run_kwargs(getattr(W, base), **over)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 22, capacity_spawns=1 << 23, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(120):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, (base, t))


def test_angle_site_dependent_guide_bitexact(ddqmc):
    """A different ratio on every site: every configuration takes the
    warp-cooperative path, whose move table holds both parts of every flip."""
    r = [0.35 + 0.07 * k for k in range(9)]
    args = (3, 3, 1, 0.9, 1.0, 1.0, 1.0, 0.01, 20000)
    kw = dict(n_a=2, control=1, seed=5, guide_kind=2, site_ratio=r, field_h=0.3, field_axis=2, field_theta=0.9)
    gpu = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(120):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


def test_angle_two_word_keys(ddqmc):
    """6x6 periodic (two-word keys, every configuration on the warp-cooperative
    path), against the oracle."""
    args = (6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 20000)
    kw = dict(n_a=3, control=1, seed=4, field_h=0.2, field_axis=2, field_theta=1.3)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 20, capacity_spawns=1 << 21, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(60):
        gpu.step(1)
        cpu.step(1)
        if t % 5 == 0 or t >= 57:
            _same(gpu, cpu, t)


def test_angle_batch_mixed_axes(ddqmc):
    """A batch whose runs have no field, a field along x, along y and at an
    angle: the runs without the angle see zero-rate y parts."""
    runs = [
        dict(Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=4000, n_a=0, seed=1),
        dict(Jx=0.8, Jy=1.0, Jz=1.0, gamma=1.5, dt=0.005, target=5000, n_a=0, seed=11, field_h=0.2),
        dict(Jx=0.9, Jy=1.2, Jz=1.0, gamma=1.0, dt=0.01, target=2000, n_a=2, seed=5, field_h=-0.3, field_axis=1),
        dict(Jx=1.1, Jy=1.0, Jz=0.7, gamma=0.6, dt=0.01, target=3000, n_a=3, seed=7, control=1, field_h=0.35,
             field_axis=2, field_theta=0.6),
    ]
    batch = ddqmc.Batch(2, 2, 0, runs)
    cpus = [O.OracleRun(2, 2, 0, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"],
                        **{k: v for k, v in r.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")})
            for r in runs]
    for t in range(100):
        batch.step(1)
        for k, cpu in enumerate(cpus):
            cpu.step(1)
            g, c = batch.export(k), cpu.export()
            assert len(g[0]) == len(c[0]), (t, k)
            for x, y in zip(g, c):
                assert np.array_equal(x, y), (t, k)
            assert np.array_equal(batch.raw_estimates(k), cpu.estimates_now()), (t, k)


def test_angle_move_table_limit(ddqmc):
    """2B + 5N moves must fit the warp-cooperative move table: 8x8 periodic
    (576 moves) is refused."""
    with pytest.raises(ddqmc.DDQMCError):
        ddqmc.Run(8, 8, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 1000, field_h=0.1, field_axis=2, field_theta=0.5)
    with pytest.raises(ddqmc.DDQMCError):
        ddqmc.Run(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.005, 1000, field_h=0.1, field_axis=3)

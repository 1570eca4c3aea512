"""GPU path (through the C-ABI) against the CPU oracle, element by element.

Walker lists (keys and int32 populations) and the integer estimator
numerators must be bit-identical after every step; the blocking moments are
exact integers and must be identical too."""
import numpy as np
import pytest

from oracle import blocking as Bk
from oracle import oracle as O
from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as d
    return d


def _pair(ddqmc, cfg, **over):
    args, kw = W.run_kwargs(cfg, **over)
    return ddqmc.Run(*args, **kw), O.OracleRun(*args, **kw)


def _same(gpu, cpu, where):
    g = gpu.export()
    c = cpu.export()
    assert len(g[0]) == len(c[0]), (where, len(g[0]), len(c[0]))
    for name, a, b in zip(("ket", "bra", "re", "im"), g, c):
        assert np.array_equal(a, b), (where, name)
    assert np.array_equal(gpu.raw_estimates(), cpu.estimates_now()), where


def test_first_steps_2x2(ddqmc):
    gpu, cpu = _pair(ddqmc, W.C1)
    for t in range(300):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)
        s, o = gpu.state(), cpu.state()
        assert s.t == o["t"] and s.shift == o["S"] and s.variable == o["variable"]


def test_c1_all_steps_bitexact(ddqmc):
    """2x2 open, seed 1: every one of the 2 x 10^4 steps."""
    gpu, cpu = _pair(ddqmc, W.C1)
    for t in range(W.C1["steps"]):
        gpu.step(1)
        cpu.step(1)
        if t % 10 == 0 or t > W.C1["steps"] - 5:
            _same(gpu, cpu, t)
    st, o = gpu.state(), cpu.state()
    assert (st.t, st.shift, st.variable, st.t_var, st.t_eq) == (o["t"], o["S"], o["variable"], o["t_var"], o["t_eq"])


def test_c2_first_200_steps_bitexact(ddqmc):
    """3x3 periodic, n_a = 3, seed 2: the first 200 steps."""
    gpu, cpu = _pair(ddqmc, W.C2)
    for t in range(200):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


VARIANTS = [
    # (base config, overrides): every one keeps its population bounded
    ("C1", dict(guide_kind=1, guide_p=3.0, dt=0.05, control=1, target=5000)),    # n_att up to 5
    ("C2", dict(guide_kind=1, guide_p=1.5, dt=0.01, control=1, target=20000)),   # uniform guide
    ("C2", dict(guide_kind=2, guide_p=0.7, n_a=2, dt=0.01, control=1, target=20000)),  # site product
    ("C1", dict(dt=0.05, shift0=25.0, n0=20000, target=10 ** 12)),               # |p_death| > 1
    ("C2", dict(Jx=0.3, Jy=-1.2, Jz=-0.7, gamma=0.6, n_a=1, seed=99, control=1, target=20000)),
    # in-plane field (Sec. V.B): single-site flips, along x and along y, with each guide
    ("C1", dict(field_h=0.3, field_axis=0)),
    ("C2", dict(field_h=-0.25, field_axis=1, guide_kind=2, guide_p=0.7, n_a=2, dt=0.01, control=1, target=20000)),
    ("C2", dict(field_h=0.4, field_axis=0, guide_kind=1, guide_p=1.5, dt=0.01, control=1, target=20000)),
    ("C3", dict(field_h=0.1, field_axis=0, target=30000)),
    ("C3", dict(field_h=-0.2, field_axis=1, target=30000, n0=5000)),
]


@pytest.mark.parametrize("base,over", VARIANTS)
def test_variants_bitexact(ddqmc, base, over):
    args, kw = W.run_kwargs(getattr(W, base), **over)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 22, capacity_spawns=1 << 23, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(120):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


@pytest.mark.parametrize("field", [0.0, 0.3])
def test_site_dependent_guide_bitexact(ddqmc, field):
    """Site-product guide with a different ratio on every site: every bond has
    its own rate table, so every configuration takes the warp-per-configuration
    path with the group-ordered cumulative table (with and without the field's
    site flips)."""
    r = [0.35 + 0.07 * k for k in range(9)]
    args = (3, 3, 1, 0.9, 1.0, 1.0, 1.0, 0.01, 20000)
    kw = dict(n_a=2, control=1, seed=5, guide_kind=2, site_ratio=r, field_h=field, field_axis=1)
    gpu = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(120):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


def test_heavy_and_light_entries_4x4(ddqmc):
    """4x4 periodic with many walkers per diagonal entry (warp-cooperative path)
    and single walkers off the diagonal (lane-per-entry path)."""
    cfg = dict(W.C3)
    cfg.update(target=3 * 10 ** 5, n0=20000)
    gpu, cpu = _pair(ddqmc, cfg)
    for t in range(60):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


@pytest.mark.parametrize("Lx,Ly,per", [(4, 5, 0), (3, 6, 1)])
def test_wide_keys_bitexact(ddqmc, Lx, Ly, per):
    """More than 16 sites: 16-byte spawn records (the packed 8-byte layout
    needs 2N <= 32), open and periodic."""
    args = (Lx, Ly, per, 0.9, 1.0, 1.0, 1.0, 0.005, 30000)
    kw = dict(n_a=3, control=1, seed=7)
    gpu = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(150):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)


TWO_WORD = [
    # (Lx, Ly, periodic, Jx, extra options): more than 31 sites
    (4, 8, 1, 0.9, {}),
    (5, 7, 0, 0.9, {}),
    (6, 6, 1, 1.1, {}),
    (6, 6, 1, 0.9, dict(guide_kind=2, site_ratio=[0.4 + 0.01 * k for k in range(36)])),
    (8, 8, 1, 0.9, {}),
    (6, 6, 1, 0.9, dict(field_h=0.2, field_axis=1)),
]


@pytest.mark.parametrize("Lx,Ly,per,Jx,extra", TWO_WORD)
def test_two_word_keys_bitexact(ddqmc, Lx, Ly, per, Jx, extra):
    """More than 31 sites (up to the 6x6 and 8x8 lattices): one 64-bit word per
    side, 24-byte records, radix digits of the ket word then of the bra word,
    128-bit merge keys, every configuration on the warp-cooperative path."""
    args = (Lx, Ly, per, Jx, 1.0, 1.0, 1.0, 0.005, 20000)
    kw = dict(n_a=3, control=1, seed=4)
    kw.update(extra)
    # the 8x8 lattice spawns about 2.7 children per walker and step
    gpu = ddqmc.Run(*args, capacity_entries=1 << 20, capacity_spawns=1 << 21, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(100):
        gpu.step(1)
        cpu.step(1)
        if t % 5 == 0 or t >= 97:
            _same(gpu, cpu, t)
    assert gpu.export()[0].size > 1000


def test_two_word_keys_larger_population(ddqmc):
    """6x6 periodic grown to 3 x 10^5 walkers, then stepped on both sides."""
    args = (6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 300000)
    kw = dict(n_a=3, control=1, seed=12, n0=20000)
    gpu = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(40):
        gpu.step(1)
        cpu.step(1)
    _same(gpu, cpu, 40)
    k, b, re, im = gpu.export()
    assert int(np.abs(re, dtype=np.int64).sum() + np.abs(im, dtype=np.int64).sum()) > 10 ** 5


@pytest.mark.parametrize("cfg", ["C1", "C3"])
def test_graph_replay_matches_single_steps(ddqmc, cfg):
    """Multi-step calls replay captured graphs of 32 steps (from either list
    buffer); they must equal step-by-step launches and the oracle."""
    over = dict(target=3 * 10 ** 4) if cfg == "C3" else {}
    args, kw = W.run_kwargs(getattr(W, cfg), **over)
    a = ddqmc.Run(*args, **kw)
    b = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    for n in (33, 64, 63, 96, 1, 31):
        a.step(n)
        for _ in range(n):
            b.step(1)
        cpu.step(n)
        for x, y in zip(a.export(), b.export()):
            assert np.array_equal(x, y), n
        _same(a, cpu, n)
        assert a.state().t == b.state().t


def test_single_step_from_imported_state(ddqmc):
    """Grow a 4x4 population on the GPU, then step the exported state once on
    both sides (the oracle imports the GPU's list and scalar state)."""
    args, kw = W.run_kwargs(W.C3, target=2 * 10 ** 6)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 25, capacity_spawns=1 << 26, **kw)
    gpu.step(1400)
    ket, bra, re, im = gpu.export()
    s = gpu.state()
    assert len(ket) > 10 ** 5
    cpu = O.OracleRun(*args, **kw)
    cpu.import_(ket, bra, re, im)
    cpu.set_state(s.t, s.shift, s.variable, s.q_prev, s.t_var, s.t_eq)
    for _ in range(2):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, "imported")


def test_blocking_moments_are_exact(ddqmc):
    """The device-resident blocking cells equal the exact block sums of the
    oracle's per-step series (same samples, integer arithmetic)."""
    gpu, cpu = _pair(ddqmc, W.C1, target=3000, t_eq=50)
    gpu.step(3000)
    cpu.step(3000)
    ser = cpu.series()
    assert len(ser) > 2000
    est = gpu.estimates()
    assert est.n_samples == len(ser)
    for k in (0, 2, 5, cpu.nobs - 4, cpu.nobs - 1):
        ref = Bk.level_moments(ser[:, k], ser[:, 0])
        got = ddqmc.ddqmc_blocking_moments(gpu.h, k)
        for l, lv in enumerate(ref):
            if lv["n"] < 1:
                break
            g = got[l]
            assert (g["n"], g["sx"], g["sxx"], g["sxy"]) == (lv["n"], lv["sx"], lv["sxx"], lv["sxy"]), (k, l)
    lay = O.observable_layout(4, 4)
    R, err, _ = Bk.blocked_ratio(ser[:, lay["sum_z"]], ser[:, 0])
    assert abs(est.mz - R / 4) < 1e-12 and abs(est.mz_err - err / 4) < 1e-9 * err


def test_empty_and_dark_states(ddqmc):
    run = ddqmc.Run(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 1000, n0=0)
    run.step(5)
    assert len(run.export()[0]) == 0
    run = ddqmc.Run(2, 2, 0, 1.0, 1.0, 0.7, 1.0, 0.01, 5000, seed=4)
    cpu = O.OracleRun(2, 2, 0, 1.0, 1.0, 0.7, 1.0, 0.01, 5000, seed=4)
    run.step(500)
    cpu.step(500)
    _same(run, cpu, "dark")
    k, b, r, i = run.export()
    assert list(k) == [0] and list(b) == [0]


def test_capacity_error_is_reported_and_sticky(ddqmc):
    run = ddqmc.Run(3, 3, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 10 ** 6, capacity_entries=4096, capacity_spawns=4096)
    with pytest.raises(ddqmc.DDQMCError) as e:
        run.step(2000)
    assert e.value.code == -3
    with pytest.raises(ddqmc.DDQMCError):
        run.step(1)


def test_invalid_arguments_rejected(ddqmc):
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.Run(2, 2, 1, 0.9, 1.0, 1.0, 1.0, 0.01, 100)       # L = 2 periodic
    assert e.value.code == -1
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.Run(9, 8, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 100)       # 72 sites: more than one word per side
    assert e.value.code == -1
    run = ddqmc.Run(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 100)
    with pytest.raises(ddqmc.DDQMCError):
        run.import_([1, 0], [0, 0], [1, 1], [0, 0], 0, 0.0)      # not in canonical order


def test_export_into_reused_buffers(ddqmc):
    """export(out=...) writes into caller buffers that are long enough and
    gives the same list as a fresh export; short buffers are not used."""
    args, kw = W.run_kwargs(W.C1)
    run = ddqmc.Run(*args, **kw)
    run.step(200)
    ref = run.export()
    m = len(ref[0])
    bufs = tuple(np.full(m + 7, 99, dtype=dt) for dt in (np.uint64, np.uint64, np.int32, np.int32))
    got = run.export(out=bufs)
    for a, b, buf in zip(ref, got, bufs):
        assert np.array_equal(a, b) and np.shares_memory(b, buf)
    short = tuple(np.zeros(1, dtype=dt) for dt in (np.uint64, np.uint64, np.int32, np.int32))
    got2 = run.export(out=short)
    assert all(np.array_equal(a, b) for a, b in zip(ref, got2)) and len(got2[0]) == m


def test_records_import_export(ddqmc):
    """The 16-byte record layout: export_records equals export (key = bra << N
    | ket); a list imported as records steps exactly as the same list imported
    as arrays and as the oracle; bad records are rejected and leave the run
    as it was; two-word keys and batches are refused."""
    args, kw = W.run_kwargs(W.C2, target=30000)
    run = ddqmc.Run(*args, **kw)
    run.step(150)
    ket, bra, re, im = run.export()
    recs = run.export_records()
    N = 9
    assert np.array_equal(recs["key"], (bra << np.uint64(N)) | ket)
    assert np.array_equal(recs["re"], re) and np.array_equal(recs["im"], im)
    s = run.state()
    st = (s.t, s.shift, s.variable, s.q_prev, s.t_var, s.t_eq)
    a = ddqmc.Run(*args, **kw)
    b = ddqmc.Run(*args, **kw)
    a.import_records(recs, *st)
    b.import_(ket, bra, re, im, *st)
    cpu = O.OracleRun(*args, **kw)
    cpu.import_(ket, bra, re, im)
    cpu.set_state(*st)
    for t in range(20):
        a.step(1)
        b.step(1)
        cpu.step(1)
        _same(a, cpu, ("records", t))
        assert np.array_equal(a.export_records(), b.export_records())
    before = a.export_records().copy()
    for bad in (recs[::-1], np.concatenate([recs, recs[-1:]])):
        with pytest.raises(ddqmc.DDQMCError) as e:
            a.import_records(bad, *st)
        assert e.value.code == -1
    zero = recs.copy()
    zero["re"][3] = 0
    zero["im"][3] = 0
    with pytest.raises(ddqmc.DDQMCError):
        a.import_records(zero, *st)
    assert np.array_equal(a.export_records(), before)
    wide = ddqmc.Run(6, 6, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 1000)
    with pytest.raises(ddqmc.DDQMCError) as e:
        wide.export_records()
    assert e.value.code == -7
    # the 12-byte records of keys of at most 32 bits
    r32 = run.export_records32()
    assert np.array_equal(r32["key"].astype(np.uint64), recs["key"])
    assert np.array_equal(r32["re"], recs["re"]) and np.array_equal(r32["im"], recs["im"])
    c = ddqmc.Run(*args, **kw)
    c.import_records32(r32, *st)
    d = ddqmc.Run(*args, **kw)
    d.import_records(recs, *st)
    for t in range(10):
        c.step(1)
        d.step(1)
        assert np.array_equal(c.export_records32(), d.export_records32()), t
        assert np.array_equal(c.raw_estimates(), d.raw_estimates()), t
    before = c.export_records32().copy()
    with pytest.raises(ddqmc.DDQMCError) as e:
        c.import_records32(r32[::-1], *st)
    assert e.value.code == -1
    assert np.array_equal(c.export_records32(), before)
    empty = ddqmc.Run(*args, **kw)
    empty.import_records32(r32[:0], *st)
    assert len(empty.export_records32()) == 0 and len(empty.export_records()) == 0
    with pytest.raises(ddqmc.DDQMCError) as e:
        ddqmc.Run(4, 5, 0, 0.9, 1.0, 1.0, 1.0, 0.005, 1000).export_records32()
    assert e.value.code == -7


def test_p40_records_split_large_counts(ddqmc):
    """4x5 open (40-bit keys: 8-byte records with 11/12-bit Delta fields):
    2x10^5 walkers on one configuration take the warp-cooperative path, whose
    per-move child counts (thousands: |Jx - Jy| = 0.7, dt = 0.02) exceed the
    fields and are split over several records; bit-exact with the oracle."""
    args = (4, 5, 0, 0.3, 1.0, 1.0, 1.0, 0.02, 10 ** 6)
    kw = dict(n_a=3, control=1, seed=21, n0=200000)
    gpu = ddqmc.Run(*args, capacity_entries=1 << 22, capacity_spawns=1 << 23, **kw)
    cpu = O.OracleRun(*args, **kw)
    for t in range(6):
        gpu.step(1)
        cpu.step(1)
        _same(gpu, cpu, t)
        if t == 0:
            ket, bra, re, im = gpu.export()
            off = (ket != 0) | (bra != 0)
            assert int(np.abs(im[off]).max()) > 1023

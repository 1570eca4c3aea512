"""A batch of runs in one walker store (run id in the key's high bits, one
spawn / sort / merge over all runs) against the same runs one at a time.

Every run of a batch must produce the walker list, integer estimator
numerators, shift and blocked estimates of the run created alone with the
same parameters: bit for bit against the CPU oracle (2x2, 3x3), and against
the single-run GPU path where the oracle would be slow (4x4 Jx sweep, 6x6
two-word keys, site-dependent guide)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as d
    return d


def _same_lists(a, b, where):
    assert len(a[0]) == len(b[0]), (where, len(a[0]), len(b[0]))
    for name, x, y in zip(("ket", "bra", "re", "im"), a, b):
        assert np.array_equal(x, y), (where, name)


# 2x2 open: different couplings, decay rates, time steps, targets, initiator
# thresholds, population controls and seeds; one run with a field along x,
# one along y (the others then run in the field instantiation with zero rates)
RUNS_2X2 = [
    dict(Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=10 ** 4, n_a=0, seed=1),
    dict(Jx=1.1, Jy=1.0, Jz=0.7, gamma=0.6, dt=0.01, target=3000, n_a=3, seed=7, control=1),
    dict(Jx=0.8, Jy=1.0, Jz=1.0, gamma=1.5, dt=0.005, target=5000, n_a=0, seed=11, field_h=0.2),
    dict(Jx=0.9, Jy=1.2, Jz=1.0, gamma=1.0, dt=0.01, target=2000, n_a=2, seed=5, field_h=-0.3, field_axis=1),
]


def test_batch_2x2_matches_the_oracle_every_step(ddqmc):
    batch = ddqmc.Batch(2, 2, 0, RUNS_2X2)
    cpus = [O.OracleRun(2, 2, 0, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"],
                        **{k: v for k, v in r.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")})
            for r in RUNS_2X2]
    for t in range(120):
        batch.step(1)
        for k, cpu in enumerate(cpus):
            cpu.step(1)
            _same_lists(batch.export(k), cpu.export(), (t, k))
            assert np.array_equal(batch.raw_estimates(k), cpu.estimates_now()), (t, k)
            s, o = batch.state(k), cpu.state()
            assert (s.t, s.shift, s.variable) == (o["t"], o["S"], o["variable"]), (t, k)
    # then whole graph blocks
    batch.step(400)
    for k, cpu in enumerate(cpus):
        cpu.step(400)
        _same_lists(batch.export(k), cpu.export(), ("block", k))
        assert np.array_equal(batch.raw_estimates(k), cpu.estimates_now()), k


def test_batch_3x3_matches_the_oracle(ddqmc):
    runs = [dict(Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=2 * 10 ** 4, n_a=3, seed=2 + k,
                 control=k % 2) for k in range(3)]
    batch = ddqmc.Batch(3, 3, 1, runs)
    cpus = [O.OracleRun(3, 3, 1, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"], n_a=r["n_a"],
                        seed=r["seed"], control=r["control"]) for r in runs]
    for t in (1, 2, 5, 20, 40):
        done = batch.state(0).t
        batch.step(t - done)
        for k, cpu in enumerate(cpus):
            cpu.step(t - done)
            _same_lists(batch.export(k), cpu.export(), (t, k))
            assert np.array_equal(batch.raw_estimates(k), cpu.estimates_now()), (t, k)


def _alone(ddqmc, Lx, Ly, per, r, **kw):
    args = (Lx, Ly, per, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"])
    rest = {k: v for k, v in r.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")}
    rest.update(kw)
    return ddqmc.Run(*args, **rest)


def _compare_alone(ddqmc, batch, Lx, Ly, per, runs, steps, **kw):
    for k, r in enumerate(runs):
        one = _alone(ddqmc, Lx, Ly, per, r, **kw)
        one.step(steps)
        _same_lists(batch.export(k), one.export(), k)
        assert np.array_equal(batch.raw_estimates(k), one.raw_estimates()), k
        a, b = batch.estimates(k), one.estimates()
        for f in ("t", "shift", "variable", "t_var", "t_eq", "n_samples", "walkers", "entries", "walker_steps"):
            assert getattr(a, f) == getattr(b, f), (k, f)
        for f in ("mz", "mz_err", "xx", "yy", "zz"):
            x, y = getattr(a, f), getattr(b, f)
            assert (np.isnan(x) and np.isnan(y)) or x == y, (k, f, x, y)
        one.close()


def test_batch_4x4_jx_sweep_matches_single_runs(ddqmc):
    """The five Jx points of the Jx sweep as one batch (4x4 periodic, total-
    population control, n_a = 3), uneven targets, each run past its target
    and accumulating samples."""
    runs = [dict(Jx=jx, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=int(t), n_a=3, seed=4 + k, control=1, t_eq=50,
                 shift0=-3.0)
            for k, (jx, t) in enumerate(zip((0.8, 0.9, 1.0, 1.1, 1.2), (2 * 10 ** 4, 5000, 10 ** 4, 3000,
                                                                       1.5 * 10 ** 4)))]
    batch = ddqmc.Batch(4, 4, 1, runs, capacity_entries=10 ** 7, capacity_spawns=2 * 10 ** 7)
    batch.step(400)
    _compare_alone(ddqmc, batch, 4, 4, 1, runs, 400, capacity_entries=4 * 10 ** 6, capacity_spawns=8 * 10 ** 6)
    assert all(batch.estimates(k).n_samples > 0 for k in range(len(runs)))
    tot = batch.totals()
    assert tot["walker_steps"] == sum(batch.estimates(k).walker_steps for k in range(len(runs)))


def test_batch_site_dependent_guide_matches_single_runs(ddqmc):
    """Site-dependent importance ratios: every configuration on the
    warp-cooperative path with per-bond rate tables."""
    ratios = [0.3 + 0.05 * k for k in range(9)]
    runs = [dict(Jx=0.9 + 0.1 * k, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=2 * 10 ** 4, n_a=3, seed=20 + k,
                 control=1) for k in range(3)]
    batch = ddqmc.Batch(3, 3, 1, runs, guide_kind=2, site_ratio=ratios)
    batch.step(150)
    _compare_alone(ddqmc, batch, 3, 3, 1, runs, 150, guide_kind=2, site_ratio=ratios)


@pytest.mark.parametrize("bits", [64, 36, -1])
def test_batch_two_word_keys_match_single_runs(ddqmc, bits):
    """6x6 periodic (36 sites): the batch in the hashed order at the default
    (for three runs 46 hash bits, one digit byte past the 36 spin and 2
    run-id bits: run id from bit 46, 6 digit passes), with 36 (run id from
    bit 36, 5 passes) and in the plain order (10 passes), against single runs
    in the hashed order."""
    runs = [dict(Jx=0.8 + 0.2 * k, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=3 * 10 ** 4, n_a=3, seed=30 + k,
                 control=1) for k in range(3)]
    batch = ddqmc.Batch(6, 6, 1, runs, capacity_entries=10 ** 7, capacity_spawns=2 * 10 ** 7, wide_sort_bits=bits)
    batch.step(80)
    _compare_alone(ddqmc, batch, 6, 6, 1, runs, 80, capacity_entries=4 * 10 ** 6, capacity_spawns=8 * 10 ** 6)


def test_batch_of_one_and_a_run_without_walkers(ddqmc):
    base = dict(Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=5000, n_a=0)
    one = ddqmc.Batch(2, 2, 0, [dict(base, seed=3)])
    one.step(64)
    _compare_alone(ddqmc, one, 2, 2, 0, [dict(base, seed=3)], 64)
    two = ddqmc.Batch(2, 2, 0, [dict(base, seed=3, n0=0), dict(base, seed=4)])
    two.step(64)
    assert two.export(0)[0].size == 0 and two.state(0).entries == 0
    alone = _alone(ddqmc, 2, 2, 0, dict(base, seed=4))
    alone.step(64)
    _same_lists(two.export(1), alone.export(), "run 1")


def test_batch_argument_checks(ddqmc):
    base = dict(Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=5000)
    with pytest.raises(ddqmc.DDQMCError) as e:      # 8x8 needs an extra key word
        ddqmc.Batch(8, 8, 1, [base, base])
    assert e.value.code == -7
    with pytest.raises(ddqmc.DDQMCError) as e:      # a bad run parameter
        ddqmc.Batch(2, 2, 0, [base, dict(base, dt=0.0)])
    assert e.value.code == -1
    b = ddqmc.Batch(2, 2, 0, [base, base])
    with pytest.raises(ddqmc.DDQMCError):           # single-run queries refuse a batch
        ddqmc.ddqmc_get_state(b.h)
    with pytest.raises(ddqmc.DDQMCError):           # no such run
        b.state(2)

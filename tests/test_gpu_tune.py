"""The launch-shape autotuner: it times candidate shapes on the run's own
list, restores the run's state after every trial, and leaves a run that
continues exactly as an untuned one (shapes never change results)."""
import math

import numpy as np
import pytest

from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as D
    return D


def _same_lists(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("cfg,target", [(W.C3, 2 * 10 ** 5), (W.C2W, 2 * 10 ** 4)])
def test_tuned_run_continues_as_untuned(ddqmc, cfg, target):
    args, kw = W.run_kwargs(cfg, target=target)
    # the population overshoots its switch-on target several times over
    kw.update(capacity_entries=16 * target + 65536, capacity_spawns=32 * target + 65536)
    a = ddqmc.Run(*args, **kw)
    b = ddqmc.Run(*args, **kw)
    a.step(300)
    b.step(300)
    t = a.tune()
    # within what each kernel can hold: spawn of packed single runs 4 blocks per SM, radix 3
    assert 1 <= t["spawn_blocks_per_sm"] <= 4 and 1 <= t["radix_blocks_per_sm"] <= 3
    assert t["heavy_walkers"] in (256, 1024, 4096)
    assert t["step_ms_tuned"] <= t["step_ms_default"] * 1.0001
    assert a.tuning()["merge_blocks_per_sm"] == t["merge_blocks_per_sm"]
    _same_lists(a.export(), b.export())
    assert np.array_equal(a.raw_estimates(), b.raw_estimates())
    sa, sb = a.state(), b.state()
    assert (sa.t, sa.shift, sa.variable, sa.q_prev) == (sb.t, sb.shift, sb.variable, sb.q_prev)
    a.step(70)                          # plain launches and then whole graphs with the new shapes
    b.step(70)
    _same_lists(a.export(), b.export())
    assert np.array_equal(a.raw_estimates(), b.raw_estimates())
    ea, eb = a.estimates(), b.estimates()
    assert ea.mz == eb.mz or (math.isnan(ea.mz) and math.isnan(eb.mz))
    # a later run of the same kind starts with the tuned shapes
    c = ddqmc.Run(*args, **kw)
    assert c.tuning()["radix_records_per_thread"] == t["radix_records_per_thread"]
    for r in (a, b, c):
        r.close()


def test_tuned_batch_continues_as_untuned(ddqmc):
    runs = [dict(Jx=0.225 + 0.01 * k, Jy=0.335, Jz=0.25, gamma=1.0, dt=0.005, target=5000 * (k + 1), n_a=0,
                 seed=90 + k, control=1) for k in range(4)]
    a = ddqmc.Batch(3, 3, 1, runs)
    b = ddqmc.Batch(3, 3, 1, runs)
    a.step(200)
    b.step(200)
    a.tune()
    a.step(64)
    b.step(64)
    for k in range(4):
        _same_lists(a.export(k), b.export(k))
        assert np.array_equal(a.raw_estimates(k), b.raw_estimates(k))
    a.close()
    b.close()

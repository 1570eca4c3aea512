"""The oracle's gathered step against its whole-list step.

``OracleRun.gather`` evaluates one step of a list only at chosen
configurations: a target's own walkers (death/clone, on-site transfer) plus
the children sent to it by every occupied configuration that can reach it
(Sec. III.C moves, reversed), under the initiator rule of Sec. IV.A.  It is
what makes full-size parity checks possible, one sampled output at a time, so
here it must reproduce the whole-list step (itself pinned by the other oracle
tests) exactly, at every occupied, vacated and empty target.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W


def _cases():
    yield "2x2 open, n_a=0", dict(W.C1), 400
    yield "3x3 periodic, n_a=3", dict(W.C2, target=3000), 300
    yield "4x4 periodic, guide, n_a=3", dict(W.C3, target=4000), 250
    yield "2x2 open, field along x", dict(W.C1, field_h=0.3, field_axis=0), 300
    yield "3x3 periodic, field along y, n_a=3", dict(W.C2, target=3000, field_h=-0.2, field_axis=1), 200


@pytest.mark.parametrize("name,cfg,steps", list(_cases()), ids=[c[0] for c in _cases()])
def test_gather_equals_step(name, cfg, steps):
    args, kw = W.run_kwargs(cfg)
    run = O.OracleRun(*args, **kw)
    run.step(steps)
    k0, b0, r0, i0 = run.export()
    st = run.state()
    run.step(1)
    k1, b1, r1, i1 = run.export()
    assert len(k0) > 20 and len(k1) > 20
    run.set_state(**st)
    # targets: every configuration before and after the step, plus empty ones
    rng = np.random.default_rng(7)
    mask = (1 << run.N) - 1
    extra_k = rng.integers(0, mask + 1, size=64, dtype=np.uint64)
    extra_b = rng.integers(0, mask + 1, size=64, dtype=np.uint64)
    tk = np.concatenate([k0, k1, extra_k, extra_b])
    tb = np.concatenate([b0, b1, extra_b, extra_b])      # extra_b twice: diagonal targets too
    gre, gim = run.gather(k0, b0, r0, i0, tk, tb)
    after = {(int(a), int(b)): (int(x), int(y)) for a, b, x, y in zip(k1, b1, r1, i1)}
    for q in range(len(tk)):
        want = after.get((int(tk[q]), int(tb[q])), (0, 0))
        assert (int(gre[q]), int(gim[q])) == want, (name, q, int(tk[q]), int(tb[q]))
    run.close()


def test_gather_detects_a_planted_change():
    """Changing one population of the input list changes the gathered values
    of that configuration and of configurations it spawns into."""
    args, kw = W.run_kwargs(dict(W.C1))
    run = O.OracleRun(*args, **kw)
    run.step(300)
    k0, b0, r0, i0 = run.export()
    r_mod = r0.copy()
    e = int(np.argmax(np.abs(r0)))
    r_mod[e] += 7
    tk, tb = k0, b0
    a = run.gather(k0, b0, r0, i0, tk, tb)
    b = run.gather(k0, b0, r_mod, i0, tk, tb)
    assert not np.array_equal(a[0], b[0]) or not np.array_equal(a[1], b[1])
    run.close()

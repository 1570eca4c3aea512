"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The 4x4 periodic workload with the importance guide and n_a = 3 is grown on
the GPU to its shift target of 10^8 walkers (about 5e8 walkers on about 9e7
configurations once the shift holds the population), exactly as the
benchmark runs it.  One more step is then checked against the oracle:

* sampled outputs, one by one: the oracle's gathered step (its own walkers,
  plus every child sent by an occupied parent, under the initiator rule;
  Sec. III.C, Sec. IV.A) at configurations drawn from the lists before and
  after the step, from the diagonal and at random, must equal the GPU list
  entry exactly (0 where the GPU list has no entry);
* properties of the whole output: keys strictly increasing, no empty entry;
* the estimator numerators (Sec. III.A) of the whole output, recomputed by the
  oracle from the exported list, must equal the GPU's exactly.
"""
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


def _keys(k, b, N):
    return (np.asarray(b, dtype=np.uint64) << np.uint64(N)) | np.asarray(k, dtype=np.uint64)


def test_bench_scale_step_against_oracle(ddqmc):
    cfg = dict(W.C3)
    target = cfg["target"]
    args, kw = W.run_kwargs(cfg)
    run = ddqmc.Run(*args, **kw, capacity_entries=int(3.2 * target) + (1 << 20),
                    capacity_spawns=int(4.5 * target) + (1 << 20))
    while True:
        run.step(25)
        st = run.state()
        if st.variable and st.t >= st.t_var + 25:
            break
    k0, b0, r0, i0 = run.export()
    st = run.state()
    run.step(1)
    k1, b1, r1, i1 = run.export()
    est_gpu = np.asarray(run.raw_estimates(), dtype=np.int64)
    run.close()
    N = cfg["Lx"] * cfg["Ly"]
    print("t %d: %d configurations, %d walkers -> %d configurations" % (
        st.t, len(k0), int(np.abs(r0, dtype=np.int64).sum() + np.abs(i0, dtype=np.int64).sum()), len(k1)))
    assert len(k0) > 10 ** 7 and int(np.abs(r0, dtype=np.int64).sum() + np.abs(i0, dtype=np.int64).sum()) > 10 ** 8

    # whole-output properties
    key1 = _keys(k1, b1, N)
    assert np.all(key1[1:] > key1[:-1])
    assert not np.any((r1 == 0) & (i1 == 0))

    # sampled outputs, gathered one by one by the oracle
    orc = O.OracleRun(*args, **kw)
    orc.set_state(t=st.t, S=st.shift, variable=st.variable, Qprev=st.q_prev, t_var=st.t_var, t_eq=st.t_eq)
    rng = np.random.default_rng(11)
    i_new = rng.choice(len(k1), size=1500, replace=False)
    i_old = rng.choice(len(k0), size=500, replace=False)
    d = rng.integers(0, 1 << N, size=100, dtype=np.uint64)
    rk = rng.integers(0, 1 << N, size=100, dtype=np.uint64)
    rb = rng.integers(0, 1 << N, size=100, dtype=np.uint64)
    tk = np.concatenate([k1[i_new], k0[i_old], d, rk])
    tb = np.concatenate([b1[i_new], b0[i_old], d, rb])
    gre, gim = orc.gather(k0, b0, r0, i0, tk, tb)
    tkey = _keys(tk, tb, N)
    pos = np.searchsorted(key1, tkey)
    pos_c = np.minimum(pos, len(key1) - 1)
    hit = key1[pos_c] == tkey
    want_re = np.where(hit, r1[pos_c], 0).astype(np.int64)
    want_im = np.where(hit, i1[pos_c], 0).astype(np.int64)
    bad = np.nonzero((gre != want_re) | (gim != want_im))[0]
    assert len(bad) == 0, [(int(tk[q]), int(tb[q]), int(gre[q]), int(want_re[q]), int(gim[q]), int(want_im[q]))
                           for q in bad[:5]]
    orc.close()

    # estimator numerators of the whole output
    orc2 = O.OracleRun(*args, **kw)
    orc2.import_(k1, b1, r1, i1)
    est_or = orc2.estimates_now()
    orc2.close()
    assert np.array_equal(est_or[:len(est_gpu)], est_gpu[:len(est_or)])

"""The NESS-solve server on the GPU: requests that arrive while others run are
admitted and stepped concurrently (each run on its own stream, grids sized
for a share of the GPU), and every request's result -- step count, blocked
M_z and its error, and the final walker list -- is identical to the same
request run alone on the whole GPU."""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import serve as S
    return S


def _requests(S):
    # the error goal is out of reach: every request runs to its step limit
    return [
        S.SolveRequest(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, 10000, n_a=0, seed=11, tol=1e-12, max_steps=1280),
        S.SolveRequest(3, 3, 1, 0.225, 0.335, 0.25, 1.0, 0.005, 20000, n_a=0, seed=12, tol=1e-12, max_steps=2560),
        S.SolveRequest(4, 4, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 50000, n_a=3, seed=13, tol=1e-12, max_steps=2560,
                       guide_kind=1, guide_p=1.0),
        S.SolveRequest(4, 5, 0, 0.9, 1.0, 1.0, 1.0, 0.005, 20000, n_a=3, seed=14, tol=1e-12, max_steps=1280),
    ]


def _same(a, b):
    return a == b or (math.isnan(a) and math.isnan(b))


def test_results_are_the_same_alone_and_in_the_mix(serve):
    S = serve
    reqs = _requests(S)
    budget = 8 << 30
    mix = S.NessServer(budget, max_active=4, chunk=64, keep_lists=True)
    t0 = time.perf_counter()
    # two requests now, two a little later, while the first two are on the GPU
    ids = [mix.submit(r, t_arrive=t0 + (0.0 if k < 2 else 0.05)) for k, r in enumerate(reqs)]
    mix.run_until_idle()
    assert mix.peak_active >= 3
    assert mix.bytes_in_use == 0
    for k, r in enumerate(reqs):
        alone = S.NessServer(budget, max_active=1, chunk=64, keep_lists=True)
        a = alone.submit(r)
        alone.run_until_idle()
        ra, rm = alone.results[a], mix.results[ids[k]]
        assert rm.error == 0 and ra.error == 0
        assert ra.steps == rm.steps == r.max_steps
        assert ra.n_samples == rm.n_samples
        assert _same(ra.mz, rm.mz) and _same(ra.mz_err, rm.mz_err)
        for x, y in zip(ra.lists, rm.lists):
            assert np.array_equal(x, y), k
    late = [mix.results[i] for i in ids[2:]]
    early = [mix.results[i] for i in ids[:2]]
    # the late arrivals started before the early ones finished
    assert min(r.t_start for r in late) < max(r.t_done for r in early)


def test_packed_requests_match_alone_and_one_matches_the_oracle(serve):
    """Compatible requests that arrive together share one batch; each result
    equals the same request served alone, and the walker list of one of them
    equals the oracle's after the same number of steps, bit for bit."""
    S = serve
    from oracle import oracle as O
    reqs = [S.SolveRequest(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, t, n_a=n_a, seed=40 + k, control=1, tol=tol,
                           min_samples=128, max_steps=ms)
            for k, (t, n_a, tol, ms) in enumerate([(4000, 0, 0.02, 1024), (8000, 3, 1e-12, 640),
                                                   (2000, 0, 0.05, 1024), (6000, 3, 1e-12, 768)])]
    budget = 4 << 30
    srv = S.NessServer(budget, max_active=4, chunk=64, keep_lists=True)
    ids = [srv.submit(r) for r in reqs]
    srv.run_until_idle()
    assert srv.batches_made == 1 and srv.bytes_in_use == 0
    for rid, r in zip(ids, reqs):
        alone = S.NessServer(budget, max_active=1, chunk=64, keep_lists=True, pack=False)
        a = alone.submit(r)
        alone.run_until_idle()
        ra, rm = alone.results[a], srv.results[rid]
        assert rm.error == 0 and ra.steps == rm.steps and ra.n_samples == rm.n_samples
        assert _same(ra.mz, rm.mz) and _same(ra.mz_err, rm.mz_err)
        for x, y in zip(ra.lists, rm.lists):
            assert np.array_equal(x, y)
    r, res = reqs[1], srv.results[ids[1]]
    cpu = O.OracleRun(r.Lx, r.Ly, r.periodic, r.Jx, r.Jy, r.Jz, r.gamma, r.dt, r.target, n_a=r.n_a, seed=r.seed,
                      control=r.control)
    cpu.step(res.steps)
    for x, y in zip(res.lists, cpu.export()):
        assert np.array_equal(x, y)


def test_batch_retire_drops_the_run_and_leaves_the_others_alone(serve):
    from paper_1802_05931_gb300 import ddqmc
    runs = [dict(Jx=0.9 + 0.05 * k, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=3000, n_a=k % 2 * 3, seed=60 + k,
                 control=1) for k in range(3)]
    b = ddqmc.Batch(2, 2, 0, runs)
    b.step(50)
    b.retire(1)
    b.step(50)
    assert len(b.export(1)[0]) == 0
    for k in (0, 2):
        kw = {x: v for x, v in runs[k].items() if x not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")}
        r = runs[k]
        one = ddqmc.Run(2, 2, 0, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"], **kw)
        one.step(100)
        for x, y in zip(one.export(), b.export(k)):
            assert np.array_equal(x, y)
        one.close()
    b.close()

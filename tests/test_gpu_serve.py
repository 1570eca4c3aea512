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

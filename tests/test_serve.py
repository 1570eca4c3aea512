"""Scheduling logic of the NESS-solve server, on the host with stand-in runs
and batches: admission by slots and by the device-memory budget, first come
first served, no admission before arrival, retirement on the error goal or
the step limit, packing of compatible requests into one batch, retirement of
batch members at their own check points."""
import math
import types

import pytest

from paper_1802_05931_gb300 import serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeRun:
    """Blocked error 1/sqrt(samples) with samples = steps - 100."""
    live = 0

    def __init__(self, req, sm_limit):
        self.req, self.t, self.closed = req, 0, False
        FakeRun.live += 1

    def step_async(self, n):
        self.t += n

    def sync(self):
        pass

    def estimates(self):
        ns = max(0, self.t - 100)
        return types.SimpleNamespace(mz=-0.5, mz_err=(1.0 / math.sqrt(ns)) if ns else float("nan"), n_samples=ns)

    def export(self):
        return ([self.t], [0], [1], [0])

    def close(self):
        self.closed = True
        FakeRun.live -= 1


def _req(target=1000, tol=0.05, max_steps=10000):
    return S.SolveRequest(2, 2, 0, 0.9, 1.0, 1.0, 1.0, 0.01, target, tol=tol, min_samples=64, max_steps=max_steps)


def _server(budget, slots, clock, chunk=32, pack=False):
    return S.NessServer(budget, max_active=slots, chunk=chunk, make_run=FakeRun, clock=clock, keep_lists=True,
                        pack=pack, make_batch=FakeBatch)


def test_retire_on_error_goal_in_whole_chunks():
    clock = FakeClock()
    srv = _server(10 ** 12, 4, clock)
    rid = srv.submit(_req(tol=0.05))          # needs 400 samples: 500 steps, rounded up to chunks
    srv.run_until_idle()
    r = srv.results[rid]
    assert r.converged and r.steps % 32 == 0 and r.n_samples >= 400 and r.steps - 32 < 500 <= r.steps
    assert r.lists[0] == [r.steps] and FakeRun.live == 0 and srv.bytes_in_use == 0


def test_step_limit_retires_unconverged():
    clock = FakeClock()
    srv = _server(10 ** 12, 4, clock)
    rid = srv.submit(_req(tol=1e-9, max_steps=300))
    srv.run_until_idle()
    r = srv.results[rid]
    assert not r.converged and r.steps == 300


def test_admission_by_slots_and_budget_first_come_first_served():
    clock = FakeClock()
    one = _req().device_bytes()
    srv = _server(2 * one + 1, 3, clock)       # memory for two runs, three slots
    ids = [srv.submit(_req(tol=0.05)) for _ in range(5)]
    starts = []
    while not srv.idle:
        srv.cycle()
        assert len(srv.active_ids()) <= 2 and srv.bytes_in_use <= 2 * one + 1
        starts += [i for i in srv.active_ids() if i not in starts]
        clock.t += 1.0
    assert starts == ids and srv.peak_active == 2
    assert all(srv.results[i].converged for i in ids)


def test_no_admission_before_arrival():
    clock = FakeClock()
    srv = _server(10 ** 12, 4, clock)
    a = srv.submit(_req(tol=0.05), t_arrive=0.0)
    b = srv.submit(_req(tol=0.05), t_arrive=5.0)
    srv.cycle()
    assert srv.active_ids() == [a]
    clock.t = 5.0
    srv.cycle()
    assert sorted(srv.active_ids()) == [a, b]      # b joins while a runs
    while not srv.idle:
        srv.cycle()
    assert srv.results[b].t_start == 5.0 and srv.results[a].t_start == 0.0


class FakeBatch:
    """Members behave as FakeRun would alone: error 1/sqrt(steps - 100)."""
    made = []

    def __init__(self, reqs, sm_limit):
        self.reqs, self.t, self.retired, self.closed = list(reqs), 0, [], False
        FakeBatch.made.append(self)

    def step_async(self, n):
        self.t += n

    def sync(self):
        pass

    def estimates(self, k):
        ns = max(0, self.t - 100)
        return types.SimpleNamespace(mz=-0.5, mz_err=(1.0 / math.sqrt(ns)) if ns else float("nan"), n_samples=ns)

    def export(self, k):
        return ([self.t], [k], [1], [0])

    def retire(self, k):
        assert k not in self.retired
        self.retired.append(k)

    def close(self):
        self.closed = True


def test_compatible_requests_share_one_batch_and_retire_at_their_own_check_points():
    FakeBatch.made = []
    clock = FakeClock()
    srv = _server(10 ** 12, 4, clock, pack=True)
    tols = [0.05, 0.1, 0.2]                      # converge at different chunks
    ids = [srv.submit(_req(tol=t)) for t in tols]
    other = srv.submit(S.SolveRequest(3, 3, 1, 0.9, 1.0, 1.0, 1.0, 0.005, 1000, tol=0.05, min_samples=64))
    limited = srv.submit(_req(tol=1e-9, max_steps=200))   # step limit between two check points
    srv.cycle()
    assert len(FakeBatch.made) == 1 and len(FakeBatch.made[0].reqs) == 4   # the 2x2 requests
    assert FakeRun.live == 1                                             # the 3x3 one alone
    srv.run_until_idle()
    b = FakeBatch.made[0]
    assert b.closed and FakeRun.live == 0 and srv.bytes_in_use == 0
    # every member but the last is retired in the batch; the last one closes it
    assert len(b.retired) == 3 and set(b.retired) <= {0, 1, 2, 3}
    # each member's result is what it would be alone
    for rid, t in zip(ids, tols):
        alone = _server(10 ** 12, 1, FakeClock())
        a = alone.submit(_req(tol=t))
        alone.run_until_idle()
        assert srv.results[rid].steps == alone.results[a].steps
        assert srv.results[rid].n_samples == alone.results[a].n_samples and srv.results[rid].converged
    assert srv.results[limited].steps == 200 and not srv.results[limited].converged
    assert srv.results[other].converged and srv.batches_made == 1


def test_batches_respect_max_batch_and_the_unit_slots():
    FakeBatch.made = []
    clock = FakeClock()
    srv = S.NessServer(10 ** 12, max_active=2, chunk=32, make_run=FakeRun, clock=clock, pack=True, max_batch=3,
                       make_batch=FakeBatch)
    ids = [srv.submit(_req(tol=0.05)) for _ in range(8)]
    srv.cycle()
    assert [len(b.reqs) for b in FakeBatch.made] == [3, 3]     # two units, two left waiting
    assert len(srv.active_ids()) == 6
    srv.run_until_idle()
    assert all(srv.results[i].converged for i in ids) and srv.bytes_in_use == 0


def test_request_larger_than_budget_is_refused():
    srv = _server(1000, 2, FakeClock())
    with pytest.raises(ValueError):
        srv.submit(_req())


def test_percentile():
    assert S.percentile([3, 1, 2], 0.5) == 2
    assert S.percentile([1, 2, 3, 4], 0.99) == pytest.approx(3.97)


class FailingRun(FakeRun):
    """A run whose device reports a capacity error after a few chunks."""

    def sync(self):
        if self.t > 64:
            from paper_1802_05931_gb300 import ddqmc
            raise ddqmc.DDQMCError(-3, "ddqmc_sync")


def test_failed_run_is_retired_with_its_error_and_frees_memory():
    clock = FakeClock()
    srv = S.NessServer(10 ** 12, max_active=2, chunk=32, make_run=FailingRun, clock=clock)
    a = srv.submit(_req(tol=1e-9, max_steps=1000))
    srv.run_until_idle()
    r = srv.results[a]
    assert r.error == -3 and not r.converged and math.isnan(r.mz)
    assert srv.bytes_in_use == 0 and FakeRun.live == 0

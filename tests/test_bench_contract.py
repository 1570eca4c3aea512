"""The benchmark's JSON lines on CPU, with stand-ins for the GPU objects.

bench.py is the interface the measurements are read through; this runs its
single-run arm and its batch arm end to end with fake runs, fake CUDA events
and a fake clock sampler, and checks every key of the lines they print
(values are meaningless here; the GPU tests and the benchmark itself give
the real ones)."""
import json
import os
import sys
import time
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3 + 1.0


class _State:
    pass


class _FakeRun:
    """Steps add fixed walker, entry and record counts; every step is 'variable'."""

    def __init__(self, *a, **k):
        self.h = self
        self.t = 0
        self.ws = 0

    def step(self, n=1):
        self.t += n
        self.ws += 1000 * n

    def step_async(self, n=1):
        self.step(n)

    def sync(self):
        pass

    def state(self, k=0):
        s = _State()
        s.variable, s.t, s.t_var, s.t_eq, s.entries, s.shift, s.q_prev = 1, self.t, 0, 0, 100, 0.5, 1000
        return s

    def export(self, k=None, out=None):
        return tuple(np.zeros(100, dtype=d) for d in (np.uint64, np.uint64, np.int32, np.int32))

    def import_(self, *a):
        pass

    def export_records(self, out=None):
        return np.zeros(100, dtype=[("key", "<u8"), ("re", "<i4"), ("im", "<i4")])

    def import_records(self, *a):
        pass

    def export_records32(self, out=None):
        return np.zeros(100, dtype=[("key", "<u4"), ("re", "<i4"), ("im", "<i4")])

    def import_records32(self, *a):
        pass

    def raw_estimates(self, k=0):
        return np.zeros(8, dtype=np.int64)

    def tune(self):
        return {"spawn_blocks_per_sm": 3, "step_ms_default": 1.0, "step_ms_tuned": 0.9}

    def tuning(self):
        return {"spawn_blocks_per_sm": 3}

    def totals(self):
        return dict(walker_steps=self.ws, entry_steps=100 * self.t, spawn_records=300 * self.t,
                    merged_entries=100 * self.t)

    def close(self):
        pass


class _Sampler:
    def __init__(self, dev):
        pass

    def start(self):
        pass

    def stop(self):
        return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


@pytest.fixture
def fake_gpu(monkeypatch):
    sys.path.insert(0, ROOT)
    import torch
    import bench
    import __graft_entry__
    from paper_1802_05931_gb300 import ddqmc
    monkeypatch.setattr(torch.cuda, "set_device", lambda i: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "Stream", lambda: types.SimpleNamespace(cuda_stream=None))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(torch.cuda, "profiler", types.SimpleNamespace(start=lambda: None, stop=lambda: None))
    monkeypatch.setattr(__graft_entry__, "build", lambda: None)
    monkeypatch.setattr(ddqmc, "Run", _FakeRun)
    monkeypatch.setattr(ddqmc, "Batch", _FakeRun)
    monkeypatch.setattr(ddqmc, "ddqmc_get_totals", lambda h: h.totals())
    monkeypatch.setattr(ddqmc, "ddqmc_set_timing", lambda h, e: None)
    monkeypatch.setattr(ddqmc, "ddqmc_get_timing",
                        lambda h: {"spawn_death": (10.0, 2), "radix_pass": (5.0, 8), "merge_partition": (0.5, 2),
                                   "merge": (4.0, 2), "finalize": (0.1, 2),
                                   "merge_compact": (0.4, 2)})
    monkeypatch.setattr(bench, "ClockSampler", _Sampler)
    arm = {"solves_per_h": 100.0, "makespan_s": 1.0, "p50_s": 0.1, "p95_s": 0.2, "p99_s": 0.3, "converged": 1,
           "errors": 0, "steps": 10, "peak_active": 1, "batches": 0}
    monkeypatch.setattr(bench, "serve_measure",
                        lambda n, t: ({k: dict(arm) for k in ("batched", "streams", "sequential")}, "fake"))
    monkeypatch.setattr(bench, "pinned_record_buffer", lambda n, dtype=None: np.empty(n, dtype=dtype or np.uint8))
    monkeypatch.setattr(bench, "pinned_list_buffers",
                        lambda n: tuple(np.empty(n, dtype=d) for d in (np.uint64, np.uint64, np.int32, np.int32)))
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda target, seconds, warmup, steps=None: (1.5e6, dict(target=int(target), walkers=1000,
                                                                                  steps=10, seconds=1.0)))
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    return bench


def _line(capsys):
    out = capsys.readouterr().out.strip().splitlines()
    return json.loads(out[-1])


def test_single_run_line_has_every_key(fake_gpu, capsys, monkeypatch):
    bench = fake_gpu
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "2", "--warmup", "3"])
    args = bench.parse()
    world, rank, local, pg = bench.dist_setup(1)
    assert bench.gpu_arm(args, world, rank, local, pg) == 0
    line = _line(capsys)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["metric"] == "walker-steps/s" and line["n_gpus"] == 1 and line["steps"] == 2
    assert "workload" in line["config"]
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] in ("alu", "hbm") and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # counters marked previous-build give no traffic
    c = bench.profile_counters()
    if not c.get((r["kernel"], "dram_bytes_per_kernel_byte"), (0, False))[1]:
        assert r["traffic"] is None
    sm = line["sort_merge"]
    for k in ("ms_per_step", "alg_min_bytes_per_step", "frac_alg_min", "kernel_bytes_per_step",
              "frac_kernel_bytes", "dram_bytes_per_step", "frac_dram"):
        assert k in sm, k
    assert sm["frac_alg_min"] <= sm["frac_kernel_bytes"]
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and "sample" in cpu
    e2e = line["e2e"]
    assert e2e["unit"] == line["unit"] and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert e2e["h2d_bytes_per_step"] == 1200 and line["e2e_arrays"]["h2d_bytes_per_step"] == 2400
    assert line["gpu_launches"] == 18
    assert set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    sv = line["serving"]
    assert sv["unit"] == "solves/h" and set(sv["arms"]) == {"batched", "streams", "sequential"}
    assert sv["vs_sequential"] == pytest.approx(1.0)
    bt = line["batch"]
    assert bt["unit"] == line["unit"] and bt["value"] > 0 and "same_walker_steps" in bt
    assert bt["batch_over_streams"] == pytest.approx(bt["value"] / bt["streams"])


def test_batch_line_has_every_key(fake_gpu, capsys, monkeypatch):
    bench = fake_gpu
    monkeypatch.setattr(sys, "argv", ["bench.py", "--batch", "3", "--lattice", "2x2", "--batch-target", "800",
                                      "--cpu-seconds", "0.3"])
    args = bench.parse()
    assert bench.batch_arm(args) == 0
    line = _line(capsys)
    for k in ("metric", "value", "unit", "steps", "warmup", "config", "arms", "kernels", "cpu_baseline",
              "gpu_launches", "same_walker_steps", "batch_over_sequential", "batch_over_streams"):
        assert k in line, k
    assert set(line["arms"]) == {"batch", "sequential", "streams"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] > 0
    assert line["gpu_launches"] == int(round(18 / 32.0 * line["steps"]))

#!/usr/bin/env python3
"""DDQMC throughput benchmark: walker-steps per second of one DDQMC step
(spawn + death/clone, onesweep radix sort, merge-path annihilation with the
initiator rule, estimators, shift update) on the 4x4 periodic XYZ lattice.

Workload: 4x4 periodic XYZ lattice (N = 16, 32 bonds), Jx = 0.9, Jy = Jz = 1,
gamma = 1, dt = 0.005, initiator threshold n_a = 3, site-product importance
guide with uniform site ratio exp(-1.5), the shift switched on when the total
population sum |re|+|im| first reaches 1.5x10^7, after which the population
overshoots and is held near 10^8 walkers, seed 3.  The run is grown from
1000 walkers on |down..down><down..down| (untimed), settles for 1000 steps
after the shift switches on, then W warm-up steps and K timed steps follow.  Every input is synthetic: the dynamics
generate the walker lists.

One JSON line on stdout (rank 0).  ``--impl reference`` times the CPU oracle
(single-threaded C) on a bounded sample of the same workload instead.
Under torchrun each rank runs an independent replica (seed + rank); the
value is the walker-steps of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "walker-steps/s"
UNIT = "walker-steps/s"
WORKLOAD = dict(Lx=4, Ly=4, periodic=1, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, n_a=3,
                guide_kind=2, guide_p=1.5, control=1, seed=3)
SWITCH_ON = 1.5e7        # total walkers at which the shift switches on (held population ~1e8)


def workload_name(target=SWITCH_ON, lattice="4x4"):
    return ("%s periodic XYZ, Jx=0.9 Jy=Jz=1 gamma=1, dt=0.005, n_a=3, site-product guide exp(-1.5), "
            "shift switched on at %.3g total walkers, seed 3" % (lattice, target))


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--target", type=float, default=SWITCH_ON,
                    help="total walkers at which the shift switches on (the population then overshoots to "
                         "about 5.7 times this and is held there)")
    ap.add_argument("--settle", type=int, default=1000, help="untimed steps after the shift switches on")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-target", type=float, default=2e4, help="shift target of the oracle sample")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--lattice", default="4x4",
                    help="Lx x Ly periodic lattice of the same workload (the benchmark line is 4x4; "
                         "6x6 and 8x8 use two-word keys)")
    ap.add_argument("--wide-sort-bits", type=int, default=64,
                    help="two-word keys: hash bits of the sort order (-1: plain order on every key bit)")
    ap.add_argument("--capacity-factor", type=float, default=3.2,
                    help="walker-list capacity per switch-on walker (spawn capacity 1.4 times that)")
    ap.add_argument("--batch", type=int, default=0,
                    help="time N runs stepped as one batch against the same runs one at a time and on "
                         "concurrent streams (walker-steps/s), instead of the single-run benchmark")
    ap.add_argument("--batch-target", type=float, default=2e5, help="largest per-run target of --batch")
    ap.add_argument("--serve", type=int, default=0,
                    help="instead: this many synthetic NESS-solve requests through the batching server, "
                         "then the same requests on streams and one at a time")
    ap.add_argument("--serve-target", type=float, default=2e5, help="largest request target of --serve")
    ap.add_argument("--serve-default", type=int, default=32,
                    help="requests of the serving measurement added to the default line (targets up to 3e5, "
                         "about 40 s for its three arms; 0: none)")
    ap.add_argument("--batch-default", type=int, default=16,
                    help="runs of the 4x4 batch measurement added to the default line (targets up to "
                         "--batch-target; batch against one at a time and streams; 0: none)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuning)")
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3"],
                    help="c3: the 4x4 benchmark (default); c1: 2x2 open, N_w target 1e4, timed after the shift "
                         "settles; c2: 3x3 periodic, N_w target 1e6, n_a 3, its first 200 steps (the window the "
                         "parity tests compare bit for bit); c1 and c2 time the GPU and the oracle on the same steps")
    return ap.parse_args()


# the small configurations: (parameters, untimed steps after the shift switches on or None, timed steps)
SMALL_WORKLOADS = {
    "c1": (dict(Lx=2, Ly=2, periodic=0, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.01, target=10 ** 4, n_a=0, seed=1,
                control=0), 1000, 2048),
    "c2": (dict(Lx=3, Ly=3, periodic=1, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005, target=10 ** 6, n_a=3, seed=2,
                control=0), None, 200),
}


def small_arm(args):
    """Walker-steps/s of c1 or c2 on the GPU (CUDA events around the timed
    steps, graph replay in blocks of 32) and of the oracle on the same steps
    (single-threaded; c1 times its first 256 of them)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1802_05931_gb300 import ddqmc
    from oracle import oracle as O
    torch.cuda.set_device(0)
    prm, settle, K = SMALL_WORKLOADS[args.workload]
    pos = (prm["Lx"], prm["Ly"], prm["periodic"], prm["Jx"], prm["Jy"], prm["Jz"], prm["gamma"], prm["dt"],
           prm["target"])
    kw = dict(n_a=prm["n_a"], seed=prm["seed"], control=prm["control"])
    stream = torch.cuda.Stream()

    def advance(run, cpu):
        if settle is None:
            return
        while True:
            run.step(32)
            st = run.state()
            if st.variable:
                break
        run.step(st.t_var + settle - st.t)
        # the oracle continues from the GPU's state (list, step, shift)
        s = run.state()
        cpu.import_(*run.export())
        cpu.set_state(s.t, s.shift, s.variable, s.q_prev, s.t_var, s.t_eq)

    gpu = ddqmc.Run(*pos, stream=stream.cuda_stream, **kw)
    cpu = O.OracleRun(*pos, **kw)
    advance(gpu, cpu)
    w0 = ddqmc.ddqmc_get_totals(gpu.h)["walker_steps"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    gpu.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ws = ddqmc.ddqmc_get_totals(gpu.h)["walker_steps"] - w0
    Kc = K if args.workload == "c2" else 256
    cws, t0 = 0, time.perf_counter()
    for _ in range(Kc):
        cws += int(cpu.estimates_now()[3])
        cpu.step(1)
    cel = time.perf_counter() - t0
    line = {"metric": METRIC, "value": ws / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": 0,
            "ms_per_step": ms / K, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "parameters": prm,
                       "timed": "steps [%d, %d)" % (gpu.state().t - K, gpu.state().t),
                       "walkers_per_step": ws / K},
            "cpu_baseline": {"value": cws / cel, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "the first %d of the same steps, %.1f s" % (Kc, cel), "host": cpu_cores_desc()}}
    gpu.close()
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- helpers
def dist_setup(n):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def reduce_max(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) < 9:
                        continue
                    try:
                        sm.append(float(p[1]))
                        mx.append(float(p[2]))
                    except ValueError:
                        continue
                    for nm, v in zip(names, p[5:9]):
                        if v.lower().startswith("active"):
                            reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_counters():
    """Per-unit ncu counters of each kernel from the committed summary
    profiles/kernel_counters.txt (lines '<kernel> <counter> <value>', with a
    fourth word 'previous-build' when the kernel's code changed after the
    capture): warp_inst_per_walker, dram_bytes_per_kernel_byte (DRAM bytes
    over the bytes the kernel must move in its layout) and, for the
    partition, dram_bytes_per_position (per merged position, entries +
    records).  Returns {(kernel, counter): (value, current)}."""
    out = {}
    path = os.path.join(ROOT, "profiles", "kernel_counters.txt")
    try:
        with open(path) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    w = line.split()
                    out[(w[0], w[1])] = (float(w[2]), len(w) < 4 or w[3] != "previous-build")
    except Exception:
        pass
    return out


def pinned_list_buffers(n):
    """Four page-locked host arrays (ket, bra, re, im) of n entries."""
    import numpy as np
    import torch
    b = tuple(torch.empty(n, dtype=dt, pin_memory=True).numpy()
              for dt in (torch.int64, torch.int64, torch.int32, torch.int32))
    return b[0].view(np.uint64), b[1].view(np.uint64), b[2], b[3]


def pinned_record_buffer(n, dtype=None):
    """A page-locked host array of n list records (RECORD_DTYPE, or the given dtype)."""
    import torch
    from paper_1802_05931_gb300 import ddqmc
    dt = ddqmc.RECORD_DTYPE if dtype is None else dtype
    return torch.empty(dt.itemsize * n, dtype=torch.uint8, pin_memory=True).numpy().view(dt)


SMS = 152                 # GB300 streaming multiprocessors
SCHEDULERS_PER_SM = 4     # warp schedulers per SM, one warp instruction issued per cycle each


# ----------------------------------------------------------------------------- oracle sample
def oracle_sample(target, seconds, warmup, steps=None):
    """Time the CPU oracle (single-threaded) on the same workload at a smaller
    shift target: grow and settle untimed, then time steps."""
    from oracle import oracle as O
    w = WORKLOAD
    site_r = [math.exp(-w["guide_p"])] * (w["Lx"] * w["Ly"])
    run = O.OracleRun(w["Lx"], w["Ly"], w["periodic"], w["Jx"], w["Jy"], w["Jz"], w["gamma"], w["dt"],
                      int(target), n_a=w["n_a"], guide_kind=w["guide_kind"], guide_p=w["guide_p"],
                      site_ratio=site_r, seed=w["seed"], control=w["control"])
    while True:
        run.step(25)
        st = run.state()
        if st["variable"] and st["t"] >= st["t_var"] + 100:
            break
    run.step(max(warmup, 1))
    ws, n, t0 = 0, 0, time.perf_counter()
    while True:
        ws += int(run.estimates_now()[3])
        run.step(1)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    W = int(run.estimates_now()[3])
    return ws / el, dict(steps=n, seconds=el, walkers=W, target=int(target))


def cpu_cores_desc():
    try:
        import platform
        return "%s, %d host cores" % (platform.processor() or platform.machine(), os.cpu_count() or 0)
    except Exception:
        return "%d host cores" % (os.cpu_count() or 0)


def reference_arm(args, world, rank, pg):
    if rank != 0:
        return 0
    rate, info = oracle_sample(args.cpu_target, args.cpu_seconds, args.warmup, steps=args.steps)
    sample = ("oracle on the bench workload with shift target %d (about %d walkers): %d timed steps "
              "after %d warm-up steps, %.1f s" % (info["target"], info["walkers"], info["steps"],
                                                   args.warmup, info["seconds"]))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": info["steps"], "warmup": args.warmup, "ms_per_step": 1e3 * info["seconds"] / info["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": workload_name(), "sample_target": info["target"]},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": cpu_cores_desc()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def gpu_arm(args, world, rank, local, pg):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    barrier(pg)
    from paper_1802_05931_gb300 import ddqmc
    w = dict(WORKLOAD)
    w["Lx"], w["Ly"] = (int(x) for x in args.lattice.lower().split("x"))
    N = w["Lx"] * w["Ly"]
    stream = torch.cuda.Stream()
    target = int(args.target)
    cf = args.capacity_factor
    run = ddqmc.Run(w["Lx"], w["Ly"], w["periodic"], w["Jx"], w["Jy"], w["Jz"], w["gamma"], w["dt"], target,
                    n_a=w["n_a"], guide_kind=w["guide_kind"], guide_p=w["guide_p"],
                    site_ratio=[math.exp(-w["guide_p"])] * N, seed=w["seed"] + rank, control=w["control"],
                    capacity_entries=int(cf * target) + (1 << 20),
                    capacity_spawns=int(1.4 * cf * target) + (1 << 20), stream=stream.cuda_stream,
                    wide_sort_bits=args.wide_sort_bits)
    # grow and settle (untimed; whole blocks of 32 steps replay a CUDA graph)
    while True:
        run.step(32)
        st = run.state()
        if st.variable:
            break
    left = st.t_var + args.settle - st.t
    if left > 0:
        run.step(left)
    # launch shapes tuned on this list (the run's state is restored after the trials)
    tuning = run.tune() if not args.no_tune else run.tuning()
    run.step(max(args.warmup, 3))
    tot0 = ddqmc.ddqmc_get_totals(run.h)
    ddqmc.ddqmc_set_timing(run.h, 1)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    barrier(pg)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # one event between steps: per-step durations for the median / p99 (the
    # total runs from the first event to the last, host gaps included)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    # the profiler range marks the timed steps for ncu --profile-from-start off
    torch.cuda.profiler.start()
    e0.record(stream)
    for k in range(args.steps):
        run.step(1)
        (evs[k] if k < args.steps - 1 else e1).record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier(pg)
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    marks = [e0] + evs + [e1]
    step_ms = sorted(marks[k].elapsed_time(marks[k + 1]) for k in range(args.steps))
    tot1 = ddqmc.ddqmc_get_totals(run.h)
    timing = ddqmc.ddqmc_get_timing(run.h)
    ddqmc.ddqmc_set_timing(run.h, 0)
    dws = tot1["walker_steps"] - tot0["walker_steps"]
    dM = tot1["entry_steps"] - tot0["entry_steps"]
    dR = tot1["spawn_records"] - tot0["spawn_records"]
    dMn = tot1["merged_entries"] - tot0["merged_entries"]
    K = args.steps
    t_max = reduce_max(pg, ms)
    ws_all = reduce_sum(pg, dws)
    value = ws_all / (t_max / 1e3)

    # Bytes per launch.  "kernel": what each kernel must move in the layout it
    # uses (8-byte packed spawn records when 2N <= 32, 16-byte records up to 31
    # sites, 24-byte beyond; list entries 16 bytes up to 31 sites, 24 beyond).
    # "alg": the method's algorithmic minimum with 16-byte records (24 above
    # 31 sites): spawn/death reads the list, writes the populations back and
    # writes the spawns; annihilation reads the spawns and the list once and
    # writes the merged list once.
    rb = 8 if 2 * N <= 32 else (16 if N <= 31 else 24)
    lb = 16 if N <= 31 else 24
    kb = {"spawn_death": ((lb + 8) * dM + rb * dR) / K,
          "radix_pass": 2 * rb * dR / K,
          "merge": (lb * (dM + dMn) + rb * dR) / K,
          # two launches a step (tile-offset scan, copy): the copy's read and
          # write of the merged list averaged over both
          "merge_compact": lb * dMn / K}
    spawn_alg = ((lb + 8) * dM + lb * dR) / K
    ann_alg = lb * (dR + dM + dMn) / K
    positions = (dM + dR) / K
    kern = {}
    tot_ms = max(sum(v[0] for v in timing.values()), 1e-30)
    peak, peak_src = peak_hbm()
    for k, (kms, n) in timing.items():
        if n:
            kern[k] = {"ms_per_launch": kms / n, "launches": n, "share": kms / tot_ms}
            if k in kb:
                kern[k]["kernel_bytes_per_launch"] = kb[k]
                kern[k]["kernel_gbs"] = kb[k] / (kms / n / 1e3) / 1e9
                kern[k]["kernel_frac"] = kern[k]["kernel_gbs"] / peak
    dom = max((k for k in kern if k in kb), key=lambda k: timing[k][0])
    # committed per-unit ncu counters of the 4x4 benchmark workload
    counters = profile_counters() if args.lattice.lower() == "4x4" else {}

    def dram(k):
        """DRAM bytes per launch of kernel k from the committed counters (None if absent or stale)."""
        if k == "merge_partition":
            r, cur = counters.get((k, "dram_bytes_per_position"), (None, False))
            return r * positions if r is not None and cur else None
        r, cur = counters.get((k, "dram_bytes_per_kernel_byte"), (None, False))
        return r * kb[k] if r is not None and cur and k in kb else None

    for k in kern:
        d = dram(k)
        if d is not None:
            kern[k]["dram_bytes_per_launch"] = d
            kern[k]["dram_frac"] = d / (kern[k]["ms_per_launch"] / 1e3) / 1e9 / peak
    walkers_per_launch = dws / K
    dms = kern[dom]["ms_per_launch"]
    traffic = dram(dom)
    hbm_src = ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s")
    ipw, ipw_cur = counters.get((dom, "warp_inst_per_walker"), (None, False))
    if dom == "spawn_death" and ipw is not None and ipw_cur:
        # issue-bound kernel: warp instructions per second against the issue
        # rate of every warp scheduler at the SM clock sampled during the run
        mhz = clocks["sm_mhz"] if clocks else 2070.0
        ach = ipw * walkers_per_launch / (dms / 1e3) / 1e9
        pk = SMS * SCHEDULERS_PER_SM * mhz * 1e6 / 1e9
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": pk, "unit": "Gwarp-inst/s",
                    "frac": ach / pk, "traffic": traffic,
                    "peak_source": "derived: %d SMs x %d schedulers x %.0f MHz (sampled SM clock)"
                                   % (SMS, SCHEDULERS_PER_SM, mhz),
                    "warp_inst_per_walker": ipw, "thread_inst_per_walker": 32.0 * ipw,
                    "counters": "ncu capture of the current kernel code (profiles/kernel_counters.txt)",
                    "alg_bytes_per_launch": spawn_alg,
                    "hbm_alg_gbs": spawn_alg / (dms / 1e3) / 1e9, "hbm_peak_gbs": peak,
                    "hbm_alg_frac": spawn_alg / (dms / 1e3) / 1e9 / peak}
    else:
        alg_dom = spawn_alg if dom == "spawn_death" else kb[dom]
        achieved = alg_dom / (dms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_source": hbm_src,
                    "alg_bytes_per_launch": alg_dom,
                    "counters": "no current instruction count for this kernel" if dom == "spawn_death" else None}
    sm_keys = ("radix_pass", "merge_partition", "merge", "merge_compact")
    sortmerge_ms = sum(timing[k][0] for k in sm_keys if k in timing) / K
    sm_s = sortmerge_ms / 1e3
    # kernel bytes a step: per-launch bytes x launches a step
    moved = sum(kb[k] * timing[k][1] / K for k in ("radix_pass", "merge", "merge_compact") if k in timing)
    sm_dram = [dram(k) for k in sm_keys]
    sm_dram_bytes = (sum(d * timing[k][1] / K for d, k in zip(sm_dram, sm_keys) if k in timing)
                     if all(d is not None for d in sm_dram) else None)
    sort_merge = {"ms_per_step": sortmerge_ms,
                  "alg_min_bytes_per_step": ann_alg,
                  "frac_alg_min": ann_alg / sm_s / 1e9 / peak,
                  "kernel_bytes_per_step": moved,
                  "frac_kernel_bytes": moved / sm_s / 1e9 / peak,
                  "dram_bytes_per_step": sm_dram_bytes,
                  "frac_dram": sm_dram_bytes / sm_s / 1e9 / peak if sm_dram_bytes else None,
                  "note": "frac_dram: DRAM bytes of the radix passes, the partition, the merge and its compaction "
                          "(committed ncu counters per unit x this run's units) over their CUDA-event time; "
                          "frac_alg_min: 16 B x (spawn records + entries read + entries written) over the same time"}
    # end to end through the C-ABI with host buffers: import, step, export,
    # estimators, every step; the list in the most compact record layout the
    # lattice allows (the e2e key: 12-byte records up to 16 sites, 16-byte
    # records up to 31) and in the four caller arrays (e2e_arrays)
    e2e, e2e_arrays = None, None
    if args.e2e_steps > 0:
        M0 = run.state().entries
        st = run.state()
        state = (st.t, st.shift, st.variable, st.q_prev, st.t_var, st.t_eq)

        def leg(mode):
            nonlocal state
            if mode == "records32":
                buf = pinned_record_buffer(int(1.25 * M0) + 1024, ddqmc.RECORD32_DTYPE)
                get = lambda: run.export_records32(out=buf)
                put = lambda lst: run.import_records32(lst, *state)
                nbytes = lambda lst: 12 * len(lst)        # key (4 B), re, im (4 B each)
                api = "ddqmc_import_records32 / ddqmc_export_records32 (12-byte records)"
            elif mode == "records":
                buf = pinned_record_buffer(int(1.25 * M0) + 1024)
                get = lambda: run.export_records(out=buf)
                put = lambda lst: run.import_records(lst, *state)
                nbytes = lambda lst: 16 * len(lst)        # key (8 B), re, im (4 B each)
                api = "ddqmc_import_records / ddqmc_export_records (16-byte records)"
            else:
                buf = pinned_list_buffers(int(1.25 * M0) + 1024)
                get = lambda: run.export(out=buf)
                put = lambda lst: run.import_(*lst, *state)
                nbytes = lambda lst: 24 * len(lst[0])     # ket, bra (8 B each), re, im (4 B each)
                api = "ddqmc_import_walkers / ddqmc_export_walkers (ket, bra, re, im arrays)"
            lst = get()
            torch.cuda.synchronize()
            barrier(pg)
            t0 = time.perf_counter()
            e_ws, h2d, d2h = 0, 0, 0
            for _ in range(args.e2e_steps):
                put(lst)
                h2d += nbytes(lst)
                run.step(1)
                e_ws += ddqmc.ddqmc_get_totals(run.h)["walker_steps"]     # import resets the totals
                lst = get()
                d2h += nbytes(lst)
                est = run.raw_estimates()
                d2h += 8 * len(est)
                st = run.state()
                state = (st.t, st.shift, st.variable, st.q_prev, st.t_var, st.t_eq)
            el = reduce_max(pg, time.perf_counter() - t0)
            e_all = reduce_sum(pg, e_ws)
            return {"value": e_all / el, "unit": UNIT, "h2d_bytes_per_step": h2d // args.e2e_steps,
                    "d2h_bytes_per_step": d2h // args.e2e_steps, "steps": args.e2e_steps, "api": api}
        nsites = w["Lx"] * w["Ly"]
        e2e_arrays = leg("arrays")
        e2e = leg("records32") if nsites <= 16 else (leg("records") if nsites <= 31 else e2e_arrays)
    st = run.state()
    est = run.raw_estimates()
    run.close()
    if rank != 0:
        return 0
    cpu = None
    if args.cpu_seconds > 0:
        rate, info = oracle_sample(args.cpu_target, args.cpu_seconds, 3)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "oracle on the bench workload with shift target %d (about %d walkers), %d steps in %.1f s"
                         % (info["target"], info["walkers"], info["steps"], info["seconds"]),
               "host": cpu_cores_desc()}
    serving = None
    if args.serve_default > 0 and world == 1:
        out, workload = serve_measure(args.serve_default, 3e5)
        b, q = out["batched"], out["sequential"]
        serving = {"metric": "NESS solves/h", "unit": "solves/h", "workload": workload,
                   "value": b["solves_per_h"], "p50_s": b["p50_s"], "p95_s": b["p95_s"], "p99_s": b["p99_s"],
                   "vs_sequential": b["solves_per_h"] / q["solves_per_h"],
                   "vs_streams": b["solves_per_h"] / out["streams"]["solves_per_h"], "arms": out}
    batch = None
    if args.batch_default > 0 and world == 1:
        t_b = time.perf_counter()
        bruns = batch_runs(args.batch_default, args.batch_target)
        res, btune, _, _ = batch_measure(ddqmc, 4, 4, bruns, 128, 512, not args.no_tune)
        rate = {k: v[1] / v[0] for k, v in res.items()}
        batch = {"metric": METRIC, "unit": UNIT,
                 "workload": "batch of %d runs, 4x4 periodic, Jx in [0.8, 1.2], targets log-spaced in "
                             "[%.3g, %.3g] total walkers, n_a 3, dt 0.005; 128 steps timed after 512"
                             % (len(bruns), args.batch_target / 8, args.batch_target),
                 "value": rate["batch"], "sequential": rate["sequential"], "streams": rate["streams"],
                 "batch_over_sequential": rate["batch"] / rate["sequential"],
                 "batch_over_streams": rate["batch"] / rate["streams"],
                 "same_walker_steps": res["batch"][1] == res["sequential"][1] == res["streams"][1],
                 "timing": "host clock around the timed steps (each call waits for the device)",
                 "seconds": time.perf_counter() - t_b}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(args.target, args.lattice), "walkers_per_step": dws / K, "entries_per_step": dM / K,
                       "spawn_records_per_step": dR / K, "shift": st.shift, "t": st.t,
                       "l2": "inputs larger than L2 (walker list and spawn buffer are GBs)",
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline,
            "sort_merge": sort_merge,
            "step_ms": {"median": statistics.median(step_ms), "p99": step_ms[min(len(step_ms) - 1,
                                                                                   int(0.99 * len(step_ms)))],
                        "min": step_ms[0], "max": step_ms[-1]},
            "kernels": kern, "cpu_baseline": cpu, "e2e": e2e, "e2e_arrays": e2e_arrays, "serving": serving, "batch": batch, "tuning": tuning,
            "gpu_launches": int(sum(v[1] for v in timing.values())), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def serve_requests(n, max_target=2e5, seed=5):
    """Synthetic solve requests: Poisson arrivals (20/s), lattice 2x2 open, 3x3
    or 4x4 periodic, Jx ~ U[0.8, 1.1], gamma ~ U[0.5, 2], target log-uniform in
    [1e4, max_target] walkers, n_a = 3, samples from 256 steps after the shift
    switches on, goal: blocked error of M_z below 0.004 within 4096 steps."""
    import numpy as np
    from paper_1802_05931_gb300 import serve as S
    rng = np.random.default_rng(seed)
    lat = [(2, 2, 0), (3, 3, 1), (4, 4, 1)]
    out, t = [], 0.0
    for k in range(n):
        t += rng.exponential(1.0 / 20.0)
        Lx, Ly, per = lat[rng.integers(0, 3)]
        req = S.SolveRequest(Lx, Ly, per, float(rng.uniform(0.8, 1.1)), 1.0, 1.0, float(rng.uniform(0.5, 2.0)),
                             0.005, int(10 ** rng.uniform(4, math.log10(max_target))), n_a=3, seed=100 + k,
                             control=1, t_eq=256, tol=0.004, min_samples=512, max_steps=4096)
        out.append((t, req))
    return out


SERVE_ARMS = (("batched", 16, True), ("streams", 16, False), ("sequential", 1, False))


def serve_measure(n, max_target):
    """The same requests through the server three ways: packed into batches
    on 16 concurrent units, on 16 concurrent streams without packing, and one
    at a time on the whole GPU.  Solves/h over the makespan (first arrival to
    last retirement) and latency percentiles (arrival to retirement)."""
    import torch
    from paper_1802_05931_gb300 import serve as S
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    reqs = serve_requests(n, max_target)
    out = {}
    for name, slots, pack in SERVE_ARMS:
        srv = S.NessServer(budget, max_active=slots, chunk=64, pack=pack)
        t0 = time.perf_counter()
        for ta, r in reqs:
            srv.submit(r, t_arrive=t0 + ta)
        srv.run_until_idle()
        span = time.perf_counter() - t0
        lat = [r.latency for r in srv.results.values()]
        out[name] = {"solves_per_h": len(reqs) / span * 3600.0, "makespan_s": span,
                     "p50_s": S.percentile(lat, 0.5), "p95_s": S.percentile(lat, 0.95),
                     "p99_s": S.percentile(lat, 0.99),
                     "converged": sum(1 for r in srv.results.values() if r.converged),
                     "errors": sum(1 for r in srv.results.values() if r.error),
                     "steps": sum(r.steps for r in srv.results.values()), "peak_active": srv.peak_active,
                     "batches": srv.batches_made}
    workload = ("%d requests, Poisson 20/s, 2x2 open / 3x3 / 4x4 periodic, Jx U[0.8,1.1], gamma U[0.5,2], "
                "target log-U[1e4,%.0e], n_a 3, M_z error goal 0.004, at most 4096 steps" % (n, max_target))
    return out, workload


def serve_arm(args):
    """Solves/h and latency percentiles of the batching server against the same
    requests served on streams without packing and one at a time."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    out, workload = serve_measure(args.serve, args.serve_target)
    b = out["batched"]
    line = {"metric": "NESS solves/h", "value": b["solves_per_h"], "unit": "solves/h", "n_gpus": 1,
            "higher_is_better": True, "p50_s": b["p50_s"], "p95_s": b["p95_s"], "p99_s": b["p99_s"],
            "data": "synthetic", "config": {"workload": workload, "units": 16, "chunk_steps": 64},
            "batched": b, "streams": out["streams"], "sequential": out["sequential"]}
    print(json.dumps(line), flush=True)
    return 0


def batch_runs(n, target, seed=40):
    """n runs of one lattice: Jx spread over [0.8, 1.2], targets log-spaced
    over [target / 8, target] (uneven sizes), total-population control, n_a 3,
    shift S0 = -3 so that every run reaches its target within the warm-up."""
    out = []
    for k in range(n):
        f = k / max(n - 1, 1)
        out.append(dict(Jx=0.8 + 0.4 * f, Jy=1.0, Jz=1.0, gamma=1.0, dt=0.005,
                        target=int(target / 8.0 * 8.0 ** ((k * 7 % n) / max(n - 1, 1))), n_a=3, seed=seed + k,
                        control=1, shift0=-3.0))
    return out


def batch_measure(ddqmc, Lx, Ly, runs, K, W, tune):
    """Walker-steps/s of the runs stepped as one batch (one walker store, one
    launch of each kernel per step for all runs) against the same runs one
    after another and on concurrent streams (each on its share of the SMs).
    Each arm takes W warm-up steps from t = 0, then K timed steps; the runs
    are identical in every arm, so each arm steps the same walkers."""
    import torch
    per = 1 if min(Lx, Ly) >= 3 else 0
    # room for the population's overshoot of its target while the shift settles
    cap = dict(capacity_entries=8 * max(r["target"] for r in runs) + 65536,
               capacity_spawns=16 * max(r["target"] for r in runs) + 65536)
    res = {}
    # one batch
    b = ddqmc.Batch(Lx, Ly, per, runs, capacity_entries=cap["capacity_entries"] * len(runs),
                    capacity_spawns=cap["capacity_spawns"] * len(runs))
    b.step(W)
    # every arm's runs take tuned launch shapes (state restored after the trials)
    batch_tuning = b.tune() if tune else None
    w0 = b.totals()["walker_steps"]
    t0 = time.perf_counter()
    b.step(K)
    res["batch"] = (time.perf_counter() - t0, b.totals()["walker_steps"] - w0)
    # per-kernel split of the batch step: 32 more steps with CUDA events around
    # each kernel class (plain launches instead of graph replay)
    ddqmc.ddqmc_set_timing(b.h, 1)
    b.step(32)
    tm = ddqmc.ddqmc_get_timing(b.h)
    ddqmc.ddqmc_set_timing(b.h, 0)
    b.close()
    launches_per_step = sum(v[1] for v in tm.values()) / 32.0
    kern = {k: {"ms_per_step": v[0] / 32.0, "launches_per_step": v[1] / 32.0} for k, v in tm.items()}
    # one after another, each on the whole GPU
    dt_seq, ws_seq = 0.0, 0
    for r in runs:
        kw = {k: v for k, v in r.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")}
        one = ddqmc.Run(Lx, Ly, per, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"], **cap, **kw)
        one.step(W)
        if tune:
            one.tune()
        w0 = ddqmc.ddqmc_get_totals(one.h)["walker_steps"]
        t0 = time.perf_counter()
        one.step(K)
        dt_seq += time.perf_counter() - t0
        ws_seq += ddqmc.ddqmc_get_totals(one.h)["walker_steps"] - w0
        one.close()
    res["sequential"] = (dt_seq, ws_seq)
    # concurrent streams, grids sized for a share of the SMs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    share = max(1, sms // len(runs))
    many = []
    for r in runs:
        kw = {k: v for k, v in r.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")}
        many.append(ddqmc.Run(Lx, Ly, per, r["Jx"], r["Jy"], r["Jz"], r["gamma"], r["dt"], r["target"],
                              sm_limit=share, **cap, **kw))
    for m in many:
        m.step_async(W)
    for m in many:
        m.sync()
    if tune:
        for m in many:
            m.tune()
    w0 = sum(ddqmc.ddqmc_get_totals(m.h)["walker_steps"] for m in many)
    t0 = time.perf_counter()
    for m in many:
        m.step_async(K)
    for m in many:
        m.sync()
    res["streams"] = (time.perf_counter() - t0, sum(ddqmc.ddqmc_get_totals(m.h)["walker_steps"] for m in many) - w0)
    for m in many:
        m.close()
    return res, batch_tuning, kern, launches_per_step


def batch_arm(args):
    """The batch measurement (batch_measure) of --batch runs as its own line,
    with the oracle timed beside it on run 0."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1802_05931_gb300 import ddqmc
    torch.cuda.set_device(0)
    Lx, Ly = (int(x) for x in args.lattice.split("x"))
    per = 1 if min(Lx, Ly) >= 3 else 0
    runs = batch_runs(args.batch, args.batch_target)
    K = max(32, (args.steps * 16 + 31) // 32 * 32)
    W = max(512, (args.warmup * 64 + 31) // 32 * 32)
    res, batch_tuning, kern, launches_per_step = batch_measure(ddqmc, Lx, Ly, runs, K, W, not args.no_tune)
    rate = {k: v[1] / v[0] for k, v in res.items()}
    # the oracle beside it: run 0 of the batch (its smallest target), grown
    # untimed for the warm-up steps, then timed for a bounded sample
    from oracle import oracle as O
    r0 = runs[0]
    cpu = O.OracleRun(Lx, Ly, per, r0["Jx"], r0["Jy"], r0["Jz"], r0["gamma"], r0["dt"], r0["target"],
                      **{k: v for k, v in r0.items() if k not in ("Jx", "Jy", "Jz", "gamma", "dt", "target")})
    cpu.step(W)
    cws, cn, c0 = 0, 0, time.perf_counter()
    while time.perf_counter() - c0 < args.cpu_seconds / 3.0:
        cws += int(cpu.estimates_now()[3])
        cpu.step(1)
        cn += 1
    cel = time.perf_counter() - c0
    cpu_line = {"value": cws / cel, "unit": "walker-steps/s", "cores": 1, "kind": "oracle",
                "sample": "run 0 of the batch (target %d) alone, %d steps after %d untimed, %.1f s" %
                          (r0["target"], cn, W, cel)}
    line = {"metric": "walker-steps/s", "value": rate["batch"], "unit": "walker-steps/s", "n_gpus": 1,
            "steps": K, "warmup": W, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "batch of %d runs, %s %s, Jx in [0.8, 1.2], targets log-spaced in "
                                   "[%.3g, %.3g] total walkers, n_a 3, dt 0.005" %
                                   (len(runs), args.lattice, "periodic" if per else "open",
                                    args.batch_target / 8, args.batch_target),
                       "timing": "host clock around the timed steps (each call waits for the device)"},
            "same_walker_steps": res["batch"][1] == res["sequential"][1] == res["streams"][1],
            "batch_tuning": batch_tuning,
            "gpu_launches": int(round(launches_per_step * K)),
            "kernels": kern, "cpu_baseline": cpu_line,
            "arms": {k: {"seconds": v[0], "walker_steps": v[1], "walker_steps_per_s": rate[k]}
                     for k, v in res.items()},
            "batch_over_sequential": rate["batch"] / rate["sequential"],
            "batch_over_streams": rate["batch"] / rate["streams"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.serve:
        return serve_arm(args)
    if args.batch:
        return batch_arm(args)
    if args.workload != "c3":
        return small_arm(args)
    world, rank, local, pg = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            return reference_arm(args, world, rank, pg)
        return gpu_arm(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

"""Continuous-batching server of steady-state (NESS) solves.

Requests (a lattice, couplings, decay, time step, target population and an
accuracy goal for M_z) arrive over time.  Each admitted request becomes a
device-resident DDQMC run with its own CUDA stream; every cycle the server
issues a chunk of steps on every active run without waiting in between, so
the runs' kernels overlap on the GPU, then checks each run's blocked error and
retires the converged ones.  Requests that arrive while others run are
admitted as soon as a slot and enough device memory are free (admission by an
HBM budget: every run's capacities are a fixed multiple of its target).

Runs are independent (counter-based random numbers keyed by the run's own
seed) and every run advances in whole chunks, so a request's result -- its
walker list, estimators and step count -- is the same whether it runs alone
or in a mix.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, List, Optional

from . import ddqmc

SMS = 152                       # streaming multiprocessors of a GB300


@dataclasses.dataclass
class SolveRequest:
    """One steady-state solve (the parameters of ddqmc_create, plus when to stop)."""
    Lx: int
    Ly: int
    periodic: int
    Jx: float
    Jy: float
    Jz: float
    gamma: float
    dt: float
    target: int
    n_a: int = 3
    seed: int = 1
    control: int = 1
    guide_kind: int = 0
    guide_p: float = 0.0
    t_eq: int = -1              # steps between the shift switching on and the first sample (< 0: library default)
    tol: float = 0.01           # goal for the blocked standard error of M_z
    min_samples: int = 256      # accumulated steps before convergence is judged
    max_steps: int = 20000      # give up (unconverged) after this many steps
    capacity_factor: float = 8.0   # list capacity = factor * target; spawn capacity twice that

    @property
    def sites(self) -> int:
        return self.Lx * self.Ly

    def capacities(self):
        m = int(self.capacity_factor * self.target) + 65536
        return m, 2 * m

    def device_bytes(self) -> int:
        """Device memory of the run: two lists and two spawn buffers, the
        merge's tile slots (one list record per merged position), plus
        look-back words, tile bounds and fixed tables."""
        m, r = self.capacities()
        rec = 24 if self.sites > 31 else 16
        tiles = (m + r) // 288 + 3
        return (2 * m * rec + 2 * r * rec + tiles * 288 * rec + (r // 1536 + 2) * 256 * 8 + 3 * tiles * 8
                + 4 * tiles + (1 << 21))


@dataclasses.dataclass
class SolveResult:
    request_id: int
    converged: bool
    steps: int
    mz: float
    mz_err: float
    n_samples: int
    t_arrive: float
    t_start: float
    t_done: float
    error: int = 0              # DDQMC_ERR_* code if the run stopped on an error
    lists: Optional[tuple] = None   # final (ket, bra, re, im) when the server keeps them

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


def _make_run(req: SolveRequest, sm_limit: int):
    m, r = req.capacities()
    return ddqmc.Run(req.Lx, req.Ly, req.periodic, req.Jx, req.Jy, req.Jz, req.gamma, req.dt, req.target,
                     n_a=req.n_a, guide_kind=req.guide_kind, guide_p=req.guide_p, seed=req.seed,
                     control=req.control, t_eq=req.t_eq, capacity_entries=m, capacity_spawns=r,
                     sm_limit=sm_limit)


class NessServer:
    """Admit, step concurrently, retire.

    hbm_budget: bytes of device memory the active runs may hold together;
    max_active: slots; chunk: steps issued per run per cycle; sm_limit: SMs
    each run's kernel grids are sized for (default: the GPU shared by the
    slots).  make_run / clock can be replaced (tests on a host without a GPU).
    """

    def __init__(self, hbm_budget: int, max_active: int = 16, chunk: int = 64, sm_limit: Optional[int] = None,
                 make_run: Optional[Callable] = None, clock: Callable[[], float] = time.perf_counter,
                 keep_lists: bool = False):
        if hbm_budget <= 0 or max_active < 1 or chunk < 1:
            raise ValueError("bad server limits")
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.chunk = int(chunk)
        self.sm_limit = int(sm_limit) if sm_limit else max(8, math.ceil(SMS / max_active))
        self._make_run = make_run or _make_run
        self._clock = clock
        self._pending: List[tuple] = []       # (arrival time, id, request), in arrival order
        self._active: List[dict] = []
        self._next_id = 0
        self.results: dict = {}
        self.bytes_in_use = 0
        self.cycles = 0
        self.peak_active = 0
        self.keep_lists = keep_lists

    # --- requests ----------------------------------------------------------------
    def submit(self, req: SolveRequest, t_arrive: Optional[float] = None) -> int:
        if req.device_bytes() > self.hbm_budget:
            raise ValueError("request needs more device memory than the whole budget")
        rid = self._next_id
        self._next_id += 1
        self._pending.append((self._clock() if t_arrive is None else t_arrive, rid, req))
        return rid

    @property
    def idle(self) -> bool:
        return not self._pending and not self._active

    # --- one scheduling cycle ---------------------------------------------------------
    def _admit(self, now: float):
        # first come, first served: a request that does not fit blocks the ones behind it
        while self._pending and len(self._active) < self.max_active:
            t_arr, rid, req = self._pending[0]
            if t_arr > now:
                break
            need = req.device_bytes()
            if self.bytes_in_use + need > self.hbm_budget:
                break
            self._pending.pop(0)
            run = self._make_run(req, self.sm_limit)
            self.bytes_in_use += need
            self._active.append(dict(id=rid, req=req, run=run, steps=0, bytes=need, t_arrive=t_arr, t_start=now))
            self.peak_active = max(self.peak_active, len(self._active))

    def _retire(self, slot: dict, est, converged: bool, now: float, error: int = 0):
        nan = float("nan")
        lists = slot["run"].export() if (self.keep_lists and not error) else None
        self.results[slot["id"]] = SolveResult(
            slot["id"], converged, slot["steps"], est.mz if est else nan, est.mz_err if est else nan,
            est.n_samples if est else 0, slot["t_arrive"], slot["t_start"], now, error, lists)
        slot["run"].close()
        self.bytes_in_use -= slot["bytes"]

    def cycle(self):
        """Admit what has arrived and fits, issue one chunk on every active run
        (all before any wait, so their kernels overlap), then retire the runs
        that converged or ran out of steps."""
        self._admit(self._clock())
        for slot in self._active:
            n = min(self.chunk, slot["req"].max_steps - slot["steps"])
            slot["run"].step_async(n)
            slot["steps"] += n
        keep = []
        for slot in self._active:
            try:
                slot["run"].sync()
                est = slot["run"].estimates()
            except ddqmc.DDQMCError as e:       # capacity or overflow: retire with the error
                self._retire(slot, None, False, self._clock(), e.code)
                continue
            req = slot["req"]
            done = est.n_samples >= req.min_samples and math.isfinite(est.mz_err) and est.mz_err <= req.tol
            if done or slot["steps"] >= req.max_steps:
                self._retire(slot, est, done, self._clock())
            else:
                keep.append(slot)
        self._active = keep
        self.cycles += 1

    def run_until_idle(self, poll: float = 0.001):
        while not self.idle:
            if not self._active and self._pending and self._pending[0][0] > self._clock():
                time.sleep(poll)        # nothing to step until the next arrival
            self.cycle()
        return self.results


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * q
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)

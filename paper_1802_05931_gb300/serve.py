"""Continuous-batching server of steady-state (NESS) solves.

Requests (a lattice, couplings, decay, time step, target population and an
accuracy goal for M_z) arrive over time.  Each admission cycle takes, first
come first served, the requests that have arrived and fit in the device
memory budget (every run's capacities are a fixed multiple of its target)
and packs those of one lattice and one guide into a single batch: one walker
store with the run id in the key's high bits, one launch of each kernel per
step for all of them (ddqmc_create_batch).  A request with no compatible
partner in its cycle becomes a run of its own.  Every batch and every lone
run has its own CUDA stream; each cycle issues a chunk of steps on all of
them before waiting on any, so their kernels overlap on the GPU.  A member
whose blocked M_z error reached its goal (or that hit its step limit) is
retired at once: its result is recorded and the batch drops its walkers
(ddqmc_batch_retire), so it costs nothing afterwards; the batch's memory is
released when its last member retires.

Runs never interact (counter-based random numbers keyed by each run's own
seed and step) and every member is judged only at its own check points
(multiples of the chunk, and its step limit), so a request's result -- its
walker list, estimators and step count -- is the same alone, in a batch, or
next to other runs.
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
    # (6x6 and larger lattices grow to millions of walkers whatever the target
    # before the shift holds them: their requests need a far larger factor)

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


def _make_batch(reqs: List[SolveRequest], sm_limit: int):
    """One batch for requests of one lattice and guide (raises DDQMCError when
    the key layout cannot hold them: the caller then runs them alone)."""
    q0 = reqs[0]
    caps = [r.capacities() for r in reqs]
    specs = [dict(Jx=r.Jx, Jy=r.Jy, Jz=r.Jz, gamma=r.gamma, dt=r.dt, target=r.target, n_a=r.n_a, seed=r.seed,
                  control=r.control, t_eq=r.t_eq) for r in reqs]
    return ddqmc.Batch(q0.Lx, q0.Ly, q0.periodic, specs, guide_kind=q0.guide_kind, guide_p=q0.guide_p,
                       capacity_entries=sum(c[0] for c in caps), capacity_spawns=sum(c[1] for c in caps),
                       sm_limit=sm_limit)


def compat_key(req: SolveRequest):
    """Requests with equal keys can share one batch (one lattice, one guide)."""
    return (req.Lx, req.Ly, req.periodic, req.guide_kind, req.guide_p)


class NessServer:
    """Admit, pack, step concurrently, retire.

    hbm_budget: bytes of device memory the active requests may hold together;
    max_active: stepping units (lone runs or batches) at once; chunk: steps
    between convergence checks; sm_limit: SMs each unit's kernel grids are
    sized for (default: the GPU shared by the units); pack: put compatible
    requests of one admission cycle into one batch (at most max_batch).
    make_run / make_batch / clock can be replaced (tests on a host without a
    GPU).
    """

    def __init__(self, hbm_budget: int, max_active: int = 16, chunk: int = 64, sm_limit: Optional[int] = None,
                 make_run: Optional[Callable] = None, clock: Callable[[], float] = time.perf_counter,
                 keep_lists: bool = False, pack: bool = True, max_batch: int = 32,
                 make_batch: Optional[Callable] = None):
        if hbm_budget <= 0 or max_active < 1 or chunk < 1 or max_batch < 1:
            raise ValueError("bad server limits")
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.chunk = int(chunk)
        self.sm_limit = int(sm_limit) if sm_limit else max(8, math.ceil(SMS / max_active))
        self._make_run = make_run or _make_run
        self._make_batch = make_batch or _make_batch
        self.pack = bool(pack)
        self.max_batch = int(max_batch)
        self._clock = clock
        self._pending: List[tuple] = []       # (arrival time, id, request), in arrival order
        self._active: List[dict] = []         # stepping units
        self._next_id = 0
        self.results: dict = {}
        self.bytes_in_use = 0
        self.cycles = 0
        self.peak_active = 0                  # most requests in progress at once
        self.batches_made = 0
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

    def active_ids(self) -> List[int]:
        return [m["id"] for u in self._active for m in u["members"] if not m["done"]]

    # --- one scheduling cycle ---------------------------------------------------------
    def _admit(self, now: float):
        # first come, first served: a request that does not fit blocks the ones behind it
        groups: dict = {}
        order: List[list] = []
        while self._pending:
            t_arr, rid, req = self._pending[0]
            if t_arr > now:
                break
            need = req.device_bytes()
            if self.bytes_in_use + need > self.hbm_budget:
                break
            key = compat_key(req) if self.pack else rid
            g = groups.get(key)
            if g is None or len(g) >= self.max_batch:
                if len(self._active) + len(order) >= self.max_active:
                    break
                g = []
                groups[key] = g
                order.append(g)
            self._pending.pop(0)
            g.append(dict(id=rid, req=req, t_arrive=t_arr, t_start=now, bytes=need, done=False))
            self.bytes_in_use += need
        for g in order:
            units = None
            if len(g) > 1:
                try:
                    units = [dict(run=self._make_batch([m["req"] for m in g], self.sm_limit), members=g,
                                  batch=True)]
                    self.batches_made += 1
                except ddqmc.DDQMCError:
                    units = None
            if units is None:
                units = [dict(run=self._make_run(m["req"], self.sm_limit), members=[m], batch=False) for m in g]
            for u in units:
                for k, m in enumerate(u["members"]):
                    m["k"] = k
                u["steps"] = 0
                u["bytes"] = sum(m["bytes"] for m in u["members"])
                self._active.append(u)
        self.peak_active = max(self.peak_active, len(self.active_ids()))

    def _member_call(self, u: dict, m: dict, what: str):
        f = getattr(u["run"], what)
        return f(m["k"]) if u["batch"] else f()

    def _retire(self, u: dict, m: dict, est, converged: bool, now: float, error: int = 0):
        nan = float("nan")
        lists = self._member_call(u, m, "export") if (self.keep_lists and not error) else None
        self.results[m["id"]] = SolveResult(
            m["id"], converged, u["steps"], est.mz if est else nan, est.mz_err if est else nan,
            est.n_samples if est else 0, m["t_arrive"], m["t_start"], now, error, lists)
        m["done"] = True
        if u["batch"] and not error and any(not x["done"] for x in u["members"]):
            u["run"].retire(m["k"])

    def _next_check(self, u: dict, m: dict) -> int:
        """The member's next check point: the next multiple of the chunk, or its step limit."""
        nxt = (u["steps"] // self.chunk + 1) * self.chunk
        return min(nxt, m["req"].max_steps)

    def cycle(self):
        """Admit what has arrived and fits, advance every unit to the next
        check point of any of its live members (all units issued before any
        wait, so their kernels overlap), then judge the members whose check
        point it is and retire those that converged or ran out of steps."""
        self._admit(self._clock())
        for u in self._active:
            live = [m for m in u["members"] if not m["done"]]
            n = min(self._next_check(u, m) for m in live) - u["steps"]
            u["run"].step_async(n)
            u["steps"] += n
        keep = []
        for u in self._active:
            live = [m for m in u["members"] if not m["done"]]
            try:
                u["run"].sync()
            except ddqmc.DDQMCError as e:       # capacity or overflow: retire every live member with the error
                for m in live:
                    self._retire(u, m, None, False, self._clock(), e.code)
                live = []
            for m in live:
                if u["steps"] % self.chunk != 0 and u["steps"] != m["req"].max_steps:
                    continue                    # not this member's check point
                try:
                    est = self._member_call(u, m, "estimates")
                except ddqmc.DDQMCError as e:
                    self._retire(u, m, None, False, self._clock(), e.code)
                    continue
                req = m["req"]
                done = est.n_samples >= req.min_samples and math.isfinite(est.mz_err) and est.mz_err <= req.tol
                if done or u["steps"] >= req.max_steps:
                    self._retire(u, m, est, done, self._clock())
            if all(m["done"] for m in u["members"]):
                u["run"].close()
                self.bytes_in_use -= u["bytes"]
            else:
                keep.append(u)
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

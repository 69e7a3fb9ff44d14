"""Serving loop: continuous batching of simulation jobs over resident lane pools.

A job asks for `n_instances` instances of one design, each simulated for
`cycles` cycles after a reset cycle, with per-instance xorshift64 stimulus
seeded from the job's seed.  For every design the server keeps one resident
pool: a simulation of `capacity` lanes (instances) created through
``rteaal_sim_create`` when its HBM footprint fits the memory budget.  A job
occupies a contiguous range of free lanes of its design's pool:

  admission   the first queued jobs whose pool has room (pools are created when
              their footprint fits what is left of the budget; idle pools of
              other designs are released to make room);
  start       ``rteaal_sim_reset_lanes`` returns the lanes to a fresh state with
              the job's seeds; their first cycle is a reset cycle
              (``reset_per_instance``), while the pool's other jobs keep running;
  rounds      every round advances every active lane of a pool by up to
              `quantum` cycles in one ``rteaal_step`` with per-lane budgets:
              jobs admitted at different times share the launches (their work
              overlaps on the device) and frozen lanes (finished or free) are
              not written;
  completion  when a job's lanes have no cycles left its register values are
              read back, its latency (completion - arrival) recorded and its
              lanes freed for the queue.

Pools of different designs are stepped one after another on one stream (the
grid forms synchronise their CTAs, which must all be resident at once).  A
step visits only its pool's live lanes -- up to the last lane with cycles
left, with a grid capped at that work -- and lanes are handed out first-fit
from the bottom, so a partly filled pool costs in proportion to its live
lanes.  The policy is host logic only; every step of the simulation runs in
the library's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    job_id: int
    design: str
    n_instances: int
    cycles: int
    seed: int
    arrival: float = 0.0                  # seconds after the start of the run
    admitted: float | None = None
    finished: float | None = None
    lane_begin: int | None = None
    result: np.ndarray | None = None      # register values [n_regs][n_instances]

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


class LaneRanges:
    """First-fit allocator of contiguous lane ranges."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.free: list[list[int]] = [[0, capacity]]       # sorted [begin, length]

    def alloc(self, n: int) -> int | None:
        for i, (b, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = [b + n, ln - n]
                return b
        return None

    def release(self, b: int, n: int):
        self.free.append([b, n])
        self.free.sort()
        merged: list[list[int]] = []
        for fb, fl in self.free:
            if merged and merged[-1][0] + merged[-1][1] == fb:
                merged[-1][1] += fl
            else:
                merged.append([fb, fl])
        self.free = merged

    @property
    def n_free(self) -> int:
        return sum(ln for _, ln in self.free)


@dataclass
class Pool:
    name: str
    sim: object
    capacity: int
    footprint: int
    lanes: LaneRanges = None
    remaining: np.ndarray = None          # cycles left per lane
    reset_next: np.ndarray = None         # leading reset cycles for the next step, per lane
    jobs: dict = field(default_factory=dict)

    def __post_init__(self):
        self.lanes = LaneRanges(self.capacity)
        self.remaining = np.zeros(self.capacity, np.int64)
        self.reset_next = np.zeros(self.capacity, np.uint32)


class Server:
    """`backend(design_name, capacity) -> sim` creates a pool simulation;
    `footprint(design_name, capacity) -> bytes` prices it."""

    def __init__(self, backend, footprint, n_regs: dict, n_inputs: dict, reg_signals: dict,
                 capacity: dict, mem_budget: int, quantum: int = 1000,
                 seeds=None, clock=time.perf_counter):
        self.backend = backend
        self.footprint = footprint
        self.n_regs, self.n_inputs, self.reg_signals = n_regs, n_inputs, reg_signals
        self.capacity = capacity
        self.mem_budget = mem_budget
        self.quantum = quantum
        self.seeds = seeds
        self.clock = clock
        self.pools: dict[str, Pool] = {}
        self.queue: list[Job] = []
        self.done: list[Job] = []
        self.rounds = 0
        self.t0 = None

    # ------------------------------------------------------------- memory
    def used(self) -> int:
        return sum(p.footprint for p in self.pools.values())

    def _pool_for(self, design: str) -> Pool | None:
        if design in self.pools:
            return self.pools[design]
        need = self.footprint(design, self.capacity[design])
        if self.used() + need > self.mem_budget:
            for name in [n for n, p in self.pools.items() if not p.jobs]:   # release idle pools
                self.pools.pop(name).sim.close()
                if self.used() + need <= self.mem_budget:
                    break
        if self.used() + need > self.mem_budget:
            return None
        sim = self.backend(design, self.capacity[design])
        self.pools[design] = Pool(design, sim, self.capacity[design], need)
        return self.pools[design]

    # ------------------------------------------------------------- scheduling
    def now(self) -> float:
        return self.clock() - self.t0

    def _admit(self):
        still = []
        for job in self.queue:
            pool = self._pool_for(job.design)
            b = pool.lanes.alloc(job.n_instances) if pool is not None else None
            if b is None:
                still.append(job)
                continue
            seeds = self.seeds(job) if self.seeds else None
            pool.sim.reset_lanes(b, job.n_instances, seeds)
            pool.remaining[b:b + job.n_instances] = job.cycles + 1      # + the reset cycle
            pool.reset_next[b:b + job.n_instances] = 1
            job.lane_begin = b
            job.admitted = self.now()
            pool.jobs[job.job_id] = job
        self.queue = still

    def _round(self):
        for pool in self.pools.values():
            if not pool.jobs:
                continue
            per = np.minimum(pool.remaining, self.quantum).astype(np.uint32)
            pool.sim.step(per, stimulus="xorshift", reset_per_instance=pool.reset_next)
            pool.remaining -= per
            pool.reset_next[:] = 0
        for pool in self.pools.values():
            if pool.jobs:
                pool.sim.sync()
        self.rounds += 1
        for pool in self.pools.values():
            for jid in [j for j, job in pool.jobs.items()
                        if not pool.remaining[job.lane_begin:job.lane_begin + job.n_instances].any()]:
                job = pool.jobs.pop(jid)
                job.result = pool.sim.read(self.reg_signals[job.design], job.lane_begin, job.n_instances)
                job.finished = self.now()
                pool.lanes.release(job.lane_begin, job.n_instances)
                self.done.append(job)

    def run(self, trace: list[Job], idle_sleep: float = 0.0005) -> list[Job]:
        """Replay `trace` (arrival times in seconds from now) until every job is done."""
        pending = sorted(trace, key=lambda j: j.arrival)
        self.t0 = self.clock()
        i = 0
        while i < len(pending) or self.queue or any(p.jobs for p in self.pools.values()):
            t = self.now()
            while i < len(pending) and pending[i].arrival <= t:
                self.queue.append(pending[i])
                i += 1
            self._admit()
            if any(p.jobs for p in self.pools.values()):
                self._round()
            elif i < len(pending):
                time.sleep(min(idle_sleep, max(0.0, pending[i].arrival - self.now())))
            elif self.queue:
                raise RuntimeError("queued jobs can never be admitted (pool larger than the memory budget?)")
        return self.done


def latency_stats(jobs: list[Job]) -> dict:
    lat = np.array([j.latency for j in jobs if j.latency is not None])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "n": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "n": int(lat.size)}


def poisson_trace(rng_seed: int, n_jobs: int, rate_hz: float, designs: list[str],
                  cycles_mu: float, cycles_sigma: float, max_instances: int,
                  cycles_cap: int | None = None) -> list[Job]:
    """Poisson arrivals, lognormal cycle counts, uniform instance counts and designs."""
    rng = np.random.default_rng(rng_seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    cyc = np.maximum(1, np.round(rng.lognormal(cycles_mu, cycles_sigma, n_jobs))).astype(np.int64)
    if cycles_cap:
        cyc = np.minimum(cyc, cycles_cap)
    inst = rng.integers(1, max_instances + 1, n_jobs)
    des = rng.integers(0, len(designs), n_jobs)
    return [Job(k, designs[int(des[k])], int(inst[k]), int(cyc[k]), seed=1000 + k, arrival=float(t[k]))
            for k in range(n_jobs)]


def build_server(netlists: dict, capacity: dict, mem_budget: int | None = None, quantum: int = 1000,
                 kernel: str = "grid", seed_fn=None, autotune: bool = False, sim_kw: dict | None = None):
    """Server over the CUDA library: one Design per netlist, pools as Sims."""
    from . import Design, Sim
    import synth  # seeded stimulus (input generator module, no simulation arithmetic)

    designs = {k: Design(v) for k, v in netlists.items()}
    if mem_budget is None:
        import torch
        free, _total = torch.cuda.mem_get_info()
        mem_budget = int(free * 0.8)

    def backend(name, cap):
        sim = Sim(designs[name], cap, kernel=kernel, **(sim_kw or {}))
        if autotune:
            sim.autotune(cycles_per_trial=1, kernels=["grid", "tile"])
        return sim

    def footprint(name, cap):
        return designs[name].footprint(cap)

    n_regs = {k: d.info["n_regs"] for k, d in designs.items()}
    n_inputs = {k: d.info["n_inputs"] for k, d in designs.items()}
    reg_signals = {k: np.arange(d.info["n_inputs"], d.info["n_inputs"] + d.info["n_regs"], dtype=np.uint32)
                   for k, d in designs.items()}
    if seed_fn is None:
        def seed_fn(job):
            return synth.xorshift_seeds(job.seed, n_inputs[job.design], job.n_instances)
    srv = Server(backend, footprint, n_regs, n_inputs, reg_signals, capacity, mem_budget, quantum, seed_fn)
    srv.designs = designs
    return srv

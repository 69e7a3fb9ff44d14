"""Benchmark: op-evaluations/s of batched cycle-accurate RTL simulation on one GB300.

Default workload ("batch-1M"): random layered DAG of 1,000,000 ops, 65,536
registers, depth 80, 32 primary inputs, 4,096 stimulus instances with per-
instance cycle budgets uniform in [1k, 100k], per-instance xorshift64
stimulus, the persistent grid kernel (launch configuration autotuned).  One
step = one pass of the whole hot path (stimulus, every layer, clock edge) for
a chunk of `--chunk` cycles over every instance that still has cycles left.
The timed window covers cycles [W*chunk, (W+K)*chunk) of the job; instances
never finish inside it (budgets >= 1,000 cycles), so every instance-cycle in
the window is active.

value       op-evals/s (active instance-cycles x ops / device time), inputs resident
e2e         same metric through the public API with host buffers: explicit
            per-cycle stimulus copied from pinned host memory each step and
            64 probed register values per instance copied back each step
roofline    dominant kernel (k_grid): algorithmic bytes per launch / launch time
cpu_baseline  the oracle on this host's cores, on a bounded sample

--impl reference  times the oracle (gate-by-gate C interpreter) as the
                  reference arm, on this host's cores, same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# the metric both arms report (op-evaluations = netlist ops x instances x cycles)
METRIC = "op-evaluations/sec (ops\u00d7instances\u00d7cycles) on 1 GB300, bit-exact, % mem roofline"

WORKLOADS = {
    # name: (spec factory, instances, cycle budget range, tile lanes)
    "batch-1M": (synth.spec_batch, 4096, (1000, 100_000)),
    "single-200k": (synth.spec_single, 1, (100_000, 100_000)),
    "tiny-2k": (synth.spec_tiny, 1, (10_000, 10_000)),
    "soc-5M": (synth.spec_soc, 1024, (20_000, 20_000)),
    "mux-1M": (synth.spec_mux, 4096, (1000, 100_000)),
    "quiet-1M": (synth.spec_quiet, 4096, (20_000, 20_000)),
}
# inputs after the reset cycle: xorshift64 every cycle, or held (the
# enable-gated modular design, whose activity then comes from its enables)
HELD_INPUTS = {"quiet-1M"}


def make_netlist(workload: str) -> synth.Netlist:
    spec = WORKLOADS[workload][0]()
    return synth.generate_modular(spec) if isinstance(spec, synth.ModularSpec) else synth.generate(spec)


def width_bytes(w: np.ndarray) -> np.ndarray:
    """Bytes per lane of a row of the compact state (1, 2, 4, 8 for widths <= 8, 16, 32, 64)."""
    w = np.asarray(w, np.int64)
    return np.select([w <= 8, w <= 16, w <= 32], [1, 2, 4], 8)


def algorithmic_bytes_per_instance_cycle(nl: synth.Netlist, lanes_sharing_meta: int) -> dict:
    """Bytes one instance-cycle must move at minimum in the compact layout: every
    operand read once and every result written once, each at its row's width
    class; per register D read + Q write; per input the xorshift state read and
    written plus the input row; per write port en/addr/data; the 20-byte op
    descriptor (16-byte operand record + 4-byte output reference) amortised
    over the lanes that share one read of it."""
    sw = width_bytes(nl.signal_widths())
    ops = float(sw[nl.args.astype(np.int64)].sum() + sw[nl.op_base:].sum())
    regs = float(sw[nl.reg_d.astype(np.int64)].sum() + sw[nl.reg_base:nl.reg_base + nl.n_regs].sum())
    inputs = float(16 * nl.n_inputs + sw[:nl.n_inputs].sum())
    memw = float(sw[nl.wport[:, 1:].astype(np.int64)].sum()) if nl.n_wports else 0.0
    meta = 20.0 * nl.n_ops / max(1, lanes_sharing_meta)
    return {"ops": ops, "regs": regs, "inputs": inputs, "mem": memw, "meta": meta,
            "total": ops + regs + inputs + memw + meta}


def live_ops(nl: synth.Netlist) -> int:
    """Ops whose value can reach state that outlives the cycle: the transitive
    fan-in cone of every register's next state and every write-port signal.
    Code generated per design (the specialised form) may drop the others from
    every cycle whose values are not stored, so a rate over all ops would count
    evaluations that never happen."""
    live = np.zeros(nl.n_signals, bool)
    live[nl.reg_d.astype(np.int64)] = True
    if nl.n_wports:
        live[nl.wport[:, 1:].reshape(-1).astype(np.int64)] = True
    args = nl.args.astype(np.int64)
    off = nl.op_argoff.astype(np.int64)
    for k in range(nl.n_ops - 1, -1, -1):        # operands precede their op
        if live[nl.op_base + k]:
            live[args[off[k]:off[k + 1]]] = True
    return int(live[nl.op_base:].sum())


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    """Hash of the sources that decide the persistent kernels' memory traffic: their
    device code (kernels.cuh, persistent.cuh, the variant tables) and the state
    layout (lower.*).  DRAM counters taken on another version do not describe this one."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2601_18140_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in ("kernels.cuh", "persistent.cuh", "lower.cpp", "lower.hpp") or (
                f.startswith("variants_") and f.endswith(".cu")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:12]


def profile_traffic(kernel_key: str) -> float | None:
    """DRAM bytes per instance-cycle from the committed ncu summary, if they were
    taken on this kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_key and parts[2] == src:
            return float(parts[1])
    return None


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows: list[list[str]] = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout
                for line in out.strip().splitlines():
                    self.rows.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self) -> dict:
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(t_ms: float, evals: float, device) -> tuple[float, float]:
    """Whole-job timing across replicas: the slowest rank's time, the sum of the work."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    ev = torch.tensor([evals], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(ev[0])


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous instance shard of one rank (replicas: no data-path exchange)."""
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi


# --------------------------------------------------------------------------- CPU
def cpu_oracle_rate(nl: synth.Netlist, n_inst: int, cycles: int, seed: int, threads: int) -> dict:
    import oracle
    o = oracle.OracleSim(nl.to_bytes(), n_inst)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n_inst)
    o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs, threads=threads)
    t0 = time.perf_counter()
    o.step(cycles, mode=oracle.STIM_XORSHIFT, xs=xs, threads=threads)
    dt = time.perf_counter() - t0
    evals = float(n_inst) * cycles * nl.n_ops
    return {"value": evals / dt, "unit": "op-evals/s", "cores": threads, "kind": "oracle",
            "seconds": dt,
            "sample": "%d instances x %d cycles of the %d-op design (after reset), %d threads"
                      % (n_inst, cycles, nl.n_ops, threads)}


def cpu_sample_size(workload: str) -> tuple[int, int]:
    return {"batch-1M": (64, 8), "single-200k": (1, 2000), "tiny-2k": (1, 10_000),
            "soc-5M": (16, 4), "mux-1M": (64, 8), "quiet-1M": (64, 8)}[workload]


def run_reference(args) -> None:
    rank, world, _ = dist_env()
    if rank != 0:
        return
    _, n_inst, _ = WORKLOADS[args.workload]
    nl = make_netlist(args.workload)
    threads = os.cpu_count() or 1
    si, sc = cpu_sample_size(args.workload)
    for _ in range(args.warmup):
        cpu_oracle_rate(nl, si, max(1, sc // 4), 7, threads)
    vals = [cpu_oracle_rate(nl, si, sc, 7, threads) for _ in range(args.steps)]
    v = float(np.mean([x["value"] for x in vals]))
    ms = float(np.mean([x["seconds"] for x in vals])) * 1e3
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "op-evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "instances": n_inst, "ops": nl.n_ops,
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "op-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------- GPU
def run_ours(args) -> None:
    import torch

    import paper_2601_18140_gb300 as rt

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    _, n_total, (clo, chi) = WORKLOADS[args.workload]
    if args.instances:
        n_total = args.instances
    nl = make_netlist(args.workload)
    run_stim = "hold" if args.workload in HELD_INPUTS else "xorshift"
    lo, hi = shard(n_total, rank, world)
    n = hi - lo
    budgets_all = synth.cycle_budgets(5, n_total, clo, chi)
    budgets = budgets_all[lo:hi].copy()
    xs_all = synth.xorshift_seeds(5, nl.n_inputs, n_total)
    xs = np.ascontiguousarray(xs_all[:, lo:hi])

    design = rt.Design(nl.to_bytes(), fuse_mux_chains=args.fuse_mux_chains)
    spec_compile_s = design.specialize() if args.kernel == "specialized" else None
    kw = dict(tile_lanes=args.tile_lanes, threads=args.threads, unroll=args.unroll,
              ctas_per_sm=args.ctas_per_sm, lanes_per_thread=args.lanes_per_thread)
    sim = rt.Sim(design, n, kernel="grid" if args.activity else args.kernel, xorshift_seed=xs,
                 expected_cycles=budgets, activity=args.activity, **kw)
    stream = torch.cuda.current_stream(dev)
    remaining = budgets.astype(np.int64).copy()

    # reset cycle (not counted)
    sim.step(1, stimulus="xorshift", reset=True)
    torch.cuda.synchronize()
    info = sim.info
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        tune_cycles = 4                              # 1-cycle trials mis-rank candidates within ~1 %
        trials = sim.autotune(cycles_per_trial=tune_cycles,
                              kernels=["grid"] if args.activity else
                              (args.tune_kernels.split(",") if args.tune_kernels else None))
        info = sim.info
        tune = {"trials": len(trials), "seconds": round(time.perf_counter() - t0, 2),
                "cycles_per_trial": tune_cycles,
                "best_ms_per_cycle": round(min(t["ms"] for t in trials) / tune_cycles, 3) if trials else None}
        if args.tune_log:
            with open(args.tune_log, "w") as f:
                json.dump(trials, f, indent=0)

    C = args.chunk

    def one_step():
        per = np.minimum(remaining, C).astype(np.uint32)
        sim.step(per, stimulus=run_stim)
        remaining[:] -= per
        return int(per.astype(np.int64).sum())

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    act0 = sim.activity() if args.activity else None
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launch_ms = []
    inst_cycles = 0
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inst_cycles += one_step()
            e1.record(stream)
            launch_ms.append((e0, e1))
        end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_ms = start.elapsed_time(end)
    step_ms = [a.elapsed_time(b) for a, b in launch_ms]
    t_max = t_ms
    evals = float(inst_cycles) * nl.n_ops
    if world > 1:
        t_max, evals = reduce_over_ranks(t_ms, evals, dev)
    value = evals / (t_max / 1e3)
    n_live = live_ops(nl) if info["kernel"] == 6 else None

    # ---- roofline of the dominant kernel (one k_tile launch per step)
    sharing = info["tile_lanes"] if info["kernel"] == 2 else n
    bpc = algorithmic_bytes_per_instance_cycle(nl, sharing)
    per_launch_bytes = bpc["total"] * (inst_cycles / args.steps)
    activity = None
    if args.activity:  # skipped items move no bytes: scale by the evaluated fraction
        ev1, sk1 = sim.activity()
        ev, sk = ev1 - act0[0], sk1 - act0[1]
        frac_eval = ev / max(1, ev + sk)
        activity = {"items_evaluated": ev, "items_skipped": sk, "evaluated_fraction": frac_eval,
                    "value_is": "equivalent rate: skipped op-evaluations (unchanged operands) are counted "
                                "as evaluated; evaluated_op_evals_per_s counts only the evaluated ones",
                    "evaluated_op_evals_per_s": value * frac_eval,
                    "item": "(op, lanes of one thread) with an active lane"}
        per_launch_bytes *= frac_eval
    avg_launch_s = float(np.mean(step_ms)) / 1e3
    peaks = measured_peaks()
    achieved = per_launch_bytes / avg_launch_s / 1e9
    kname = {1: "k_layer_ops", 2: "k_tile", 3: "k_grid", 4: "k_layer_ops", 5: "k_stream",
             6: "rteaal_spec", 7: "k_cluster", 8: "k_flow"}[info["kernel"]]
    # DRAM bytes per instance-cycle of this kernel on this workload (from an ncu
    # capture of one of its launch configurations; every configuration moves the
    # same rows, only L2 reuse differs)
    traffic = profile_traffic(kname + ":" + args.workload) if n_total == WORKLOADS[args.workload][1] else None
    if traffic is not None:
        traffic *= (inst_cycles / args.steps)                # stored per instance-cycle

    # ---- sampled parity of the timed run against the oracle (bit-exact)
    parity = None
    if args.verify and rank == 0:
        import oracle
        run_cycles = budgets.astype(np.int64) - remaining
        sample = np.array(sorted({0, n // 3, n - 1}), np.int64)
        o = oracle.OracleSim(nl.to_bytes(), sample.size)
        oxs = np.ascontiguousarray(xs[:, sample])
        o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=os.cpu_count() or 1)
        o.step(run_cycles[sample].astype(np.uint32),
               mode=oracle.STIM_HOLD if run_stim == "hold" else oracle.STIM_XORSHIFT, xs=oxs,
               threads=os.cpu_count() or 1)
        live = design.present_signals()           # every signal unless fusion absorbed some
        ok = all(np.array_equal(sim.read(live, int(i), 1)[:, 0], o.vals[k][live])
                 for k, i in enumerate(sample))
        parity = ("bit-exact" if ok else "MISMATCH") + " on instances %s after %s cycles" % (
            list(map(int, sample)), list(map(int, run_cycles[sample])))
        if not ok:
            print("PARITY FAILURE", parity, file=sys.stderr)

    # ---- e2e through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        probes = (nl.reg_base + np.arange(min(64, nl.n_regs))).astype(np.uint32)
        vals_host = torch.empty((C, nl.n_inputs, n), dtype=torch.int64).pin_memory()
        vals_np = vals_host.numpy().view(np.uint64)
        if run_stim == "hold":   # the testbench drives the values the inputs hold
            vals_np[:] = sim.read(np.arange(nl.n_inputs))[None, :, :]
        else:
            vals_np[:] = synth.stimulus_values(9, C, nl.n_inputs, n)
        out_host = torch.empty((1, probes.size, n), dtype=torch.int64).pin_memory()
        e2e_evals = 0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            per = np.minimum(remaining, C).astype(np.uint32)
            cyc = rt.rteaal_cycles()
            cyc.per_instance = per.ctypes.data_as(rt.ctypes.POINTER(rt.ctypes.c_uint32))
            st = rt.rteaal_stimulus()
            st.mode, st.values, st.values_on_host = rt.RTEAAL_STIM_BUFFER, vals_host.data_ptr(), 1
            pr = rt.rteaal_probes()
            pr.signals = probes.ctypes.data_as(rt.ctypes.POINTER(rt.ctypes.c_uint32))
            pr.n, pr.mode, pr.out, pr.out_on_host = probes.size, rt.RTEAAL_PROBE_LAST, out_host.data_ptr(), 1
            rt.rteaal_step(sim.handle, cyc, st, pr, 0, stream)
            remaining[:] -= per
            e2e_evals += int(per.astype(np.int64).sum()) * nl.n_ops
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:   # whole job: the slowest rank's time, every rank's work
            e2e_ms, e2e_evals = reduce_over_ranks(e2e_s * 1e3, float(e2e_evals), dev)
            e2e_s = e2e_ms / 1e3
        e2e = {"value": e2e_evals / e2e_s, "unit": "op-evals/s",
               "h2d_bytes_per_step": int(C * nl.n_inputs * n_total * 8 + n_total * 4),   # all ranks
               "d2h_bytes_per_step": int(probes.size * n_total * 8)}

    # ---- the whole job: with uneven budgets instances retire as the job goes on
    # and each step visits only the live lanes, so the device time per cycle
    # falls with the live count.  Measure it at points t of the job (instances
    # with budget > t run a window of C cycles from their state; the others are
    # done), integrate over t, and divide the job's op-evaluations by it.
    job = None
    if args.job_points > 0:
        tmax = int(budgets_all.max())
        pts = [int(round(tmax * i / args.job_points)) for i in range(args.job_points)]
        samples = []
        for t in pts:
            per = np.clip(budgets.astype(np.int64) - t, 0, C).astype(np.uint32)
            if per.max() == 0:
                samples.append({"t": t, "live": 0, "ms_per_cycle": 0.0})
                continue
            sim.step(per, stimulus=run_stim)                     # warm-up at this span
            j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            j0.record(stream)
            for _ in range(2):
                sim.step(per, stimulus=run_stim)
            j1.record(stream)
            torch.cuda.synchronize()
            ms = j0.elapsed_time(j1) / (2 * C)
            samples.append({"t": t, "live": int((per > 0).sum()), "ms_per_cycle": ms,
                            "span": int(sim.info["last_span"]),
                            "op_evals_per_s": float(per.astype(np.int64).sum()) * nl.n_ops / (ms * C / 1e3)})
        ts = np.array([x["t"] for x in samples] + [tmax], np.float64)
        ys = np.array([x["ms_per_cycle"] for x in samples] + [0.0], np.float64)
        job_ms = float(np.sum((ys[1:] + ys[:-1]) * np.diff(ts)) / 2.0)     # trapezoid over t
        job_evals = float(budgets.astype(np.int64).sum()) * nl.n_ops
        if world > 1:
            job_ms, job_evals = reduce_over_ranks(job_ms, job_evals, dev)
        job = {"value": job_evals / (job_ms / 1e3), "unit": "op-evals/s",
               "job_seconds": job_ms / 1e3, "op_evals": job_evals,
               "over_value": (job_evals / (job_ms / 1e3)) / value,
               "method": "device time per cycle measured at %d points of the job (window of %d cycles "
                         "for the instances still running), integrated over the job's %d cycles"
                         % (len(pts), C, tmax),
               "points": samples}

    # the plain single-instance form on the same design (the batching baseline):
    # one instance, one launch sequence per cycle replayed as a CUDA graph
    plain = None
    if rank == 0 and world == 1 and args.plain_cycles > 0:
        p_sim = rt.Sim(design, 1, kernel="layer_graph", xorshift_seed=np.ascontiguousarray(xs[:, :1]))
        p_sim.step(1, stimulus="xorshift", reset=True)
        p_sim.step(2, stimulus="xorshift")                   # warm-up (graph capture)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        p_sim.step(args.plain_cycles, stimulus="xorshift", stream=stream)
        p1.record(stream)
        torch.cuda.synchronize()
        p_rate = args.plain_cycles * nl.n_ops / (p0.elapsed_time(p1) / 1e3)
        plain = {"form": "layer_graph, 1 instance", "value": p_rate, "unit": "op-evals/s",
                 "cycles": args.plain_cycles, "batched_over_plain": value / p_rate}
        p_sim.close()
        # the same instance in the FLOW form (no barrier between layers): the
        # fastest one-instance form, beside the plain one
        f_sim = rt.Sim(design, 1, kernel="flow", xorshift_seed=np.ascontiguousarray(xs[:, :1]))
        f_sim.step(1, stimulus="xorshift", reset=True)
        f_sim.step(2, stimulus="xorshift")
        torch.cuda.synchronize()
        p0.record(stream)
        f_sim.step(args.plain_cycles, stimulus="xorshift", stream=stream)
        p1.record(stream)
        torch.cuda.synchronize()
        f_rate = args.plain_cycles * nl.n_ops / (p0.elapsed_time(p1) / 1e3)
        plain["flow_one_instance"] = {"value": f_rate, "over_plain": f_rate / p_rate,
                                      "batched_over_flow": value / f_rate}
        f_sim.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        si, sc = cpu_sample_size(args.workload)
        cpu = cpu_oracle_rate(nl, si, sc, 7, os.cpu_count() or 1)
        cpu.pop("seconds", None)
        one = cpu_oracle_rate(nl, max(1, si // 16), sc, 7, 1)     # the same oracle on one core
        cpu["single_core"] = {"value": one["value"], "sample": one["sample"]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "op-evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "ops": nl.n_ops, "regs": nl.n_regs,
                       "layers": design.info["n_layers"], "instances": n_total,
                       "fused_mux_ops": design.info["n_fused"], "activity_aware": bool(args.activity),
                       "specialize_compile_s": spec_compile_s,
                       "inputs_after_reset": run_stim,
                       "cycles_per_step": C, "kernel": args.kernel,
                       "kernel_used": {1: "layer", 2: "tile", 3: "grid", 4: "layer_graph", 5: "stream",
                                       6: "specialized", 7: "cluster", 8: "flow"}[info["kernel"]],
                       "tile_lanes": info["tile_lanes"], "threads": info["threads"],
                       "ctas_per_sm": info["ctas_per_sm"], "unroll": info["unroll"],
                       "lanes_per_thread": info["lanes_per_thread"],
                       "grid": info["grid"], "autotune": tune, "parallelism": "replicas" if world > 1 else "1 gpu",
                       "l2": ("state %.1f GB >> 129 MB L2 (no flush needed)"
                              % (design.info["state_bytes_per_lane"] * n / 1e9)
                              if design.info["state_bytes_per_lane"] * n > 129e6 else
                              "state %.1f MB fits L2 and is not flushed (a latency-bound one-instance "
                              "configuration)" % (design.info["state_bytes_per_lane"] * n / 1e6))},
            "roofline": ({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                          "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                          "traffic": traffic, "peak_source": peaks["source"],
                          "bytes_per_instance_cycle": bpc["total"],
                          "kernel": kname} if info["kernel"] != 6 else
                         {"bound": "alu", "achieved": None, "peak": None, "frac": None, "kernel": kname,
                          "note": "straight-line code per instance: the state moves once per step, the "
                                  "kernel is bound by instruction issue"}),
            "gpu_launches": 1 * args.steps,
            "activity": activity,
            "specialized": ({"live_ops": n_live, "ops": nl.n_ops,
                             "value_counting_live_ops": value * ((n_live * (C - 1) + nl.n_ops) / (C * nl.n_ops)),
                             "note": "straight-line code stores every row in the last cycle of a step only, so "
                                     "ops outside the live cone may be dropped from the other cycles; this rate "
                                     "counts the live ops every cycle and all ops in the last"}
                            if info["kernel"] == 6 else None),
            "plain_single_instance": plain,
            "job": job,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "parity": parity,
        }
        print(json.dumps(line))
    sim.close()
    design.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args) -> None:
    """Serving trace: Poisson arrivals over three designs, continuous batching."""
    import torch

    from paper_2601_18140_gb300.serve import Job, build_server, latency_stats, poisson_trace

    torch.cuda.set_device(0)
    sizes = {"d50k": 50_000, "d500k": 500_000, "d5M": 5_000_000}
    nls = {k: synth.generate(synth.spec_serving(v, seed=40 + i)) for i, (k, v) in enumerate(sizes.items())}
    # pools sized to hold a saturated queue of 1-64-instance jobs of each design
    capacity = {"d50k": 2048, "d500k": 1024, "d5M": 512}
    pool_kw = ({"kernel": "stream"} if args.kernel == "stream" else
               {"kernel": "grid", "sim_kw": dict(threads=224, ctas_per_sm=4, lanes_per_thread=8)})
    srv = build_server({k: v.to_bytes() for k, v in nls.items()}, capacity, quantum=args.quantum,
                       autotune=args.serve_autotune, **pool_kw)
    warm = [Job(10_000 + i, k, 1, 10, seed=1, arrival=0.0) for i, k in enumerate(sizes)]
    srv.run(warm)
    srv.done.clear()
    trace = poisson_trace(4, args.serve_jobs, args.serve_rate, list(sizes), np.log(1e4), 1.0, 64,
                          cycles_cap=args.cycles_cap or None)
    t0 = time.perf_counter()
    with ClockSampler(0) as clk:
        done = srv.run(trace)
    wall = time.perf_counter() - t0
    work = float(sum(j.n_instances * j.cycles * nls[j.design].n_ops for j in done))
    span = max(j.arrival for j in trace)
    st = latency_stats(done)
    line = {"metric": "served op-evaluations/sec, continuous batching, p50/p99 job latency",
            "value": work / wall, "unit": "op-evals/s", "n_gpus": 1, "steps": len(done), "warmup": len(warm),
            "ms_per_step": wall * 1e3 / max(1, len(done)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "serving", "designs_ops": list(sizes.values()), "jobs": len(done),
                       "rate_hz": args.serve_rate, "cycles": "lognormal(ln 10k, 1)" +
                       (" capped at %d" % args.cycles_cap if args.cycles_cap else ""),
                       "instances": "U{1..64}", "capacity_lanes": capacity, "quantum": args.quantum,
                       "pool_autotune": bool(args.serve_autotune)},
            "latency": st, "offered_op_evals_per_s": work / max(span, 1e-9),
            "served_op_evals_per_s": work / wall, "wall_s": wall, "rounds": srv.rounds,
            "clocks": clk.summary()}
    if args.serve_load > 0:
        # the same job distribution at a Poisson rate that offers `serve_load` of the
        # capacity just measured (work per second served at saturation)
        trace2 = poisson_trace(5, args.serve_jobs, 1.0, list(sizes), np.log(1e4), 1.0, 64,
                               cycles_cap=args.cycles_cap or None)
        # stretch the arrivals so that this trace's own work arrives at the target load
        w2 = float(sum(j.n_instances * j.cycles * nls[j.design].n_ops for j in trace2))
        span2 = w2 / (args.serve_load * (work / wall))
        last = max(j.arrival for j in trace2)
        for j in trace2:
            j.arrival *= span2 / last
        rate = len(trace2) / span2
        srv.done.clear()
        t1 = time.perf_counter()
        done2 = srv.run(trace2)
        wall2 = time.perf_counter() - t1
        work2 = float(sum(j.n_instances * j.cycles * nls[j.design].n_ops for j in done2))
        line["sub_saturation"] = {
            "load_target": args.serve_load, "rate_hz": rate, "jobs": len(done2),
            "offered_op_evals_per_s": work2 / max(max(j.arrival for j in trace2), 1e-9),
            "served_op_evals_per_s": work2 / wall2, "latency": latency_stats(done2), "wall_s": wall2}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch-1M", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--serve-jobs", type=int, default=120)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-load", type=float, default=0.0,
                    help="serving: also replay a trace offering this fraction of the measured capacity")
    ap.add_argument("--quantum", type=int, default=2000)
    ap.add_argument("--serve-autotune", action="store_true",
                    help="serving: autotune each pool's launch configuration when it is created")
    ap.add_argument("--cycles-cap", type=int, default=10_000,
                    help="serving: cap on the lognormal cycle counts (0: none); stated in the line")
    ap.add_argument("--kernel", default="tile")
    ap.add_argument("--plain-cycles", type=int, default=20,
                    help="cycles of the plain single-instance form timed for comparison (0: skip)")
    ap.add_argument("--activity", action="store_true",
                    help="activity-aware evaluation (grid kernel): skip ops whose operands did not change")
    ap.add_argument("--fuse-mux-chains", action="store_true",
                    help="fuse single-fanout mux chains into one op (ops are still counted as in the netlist)")
    ap.add_argument("--chunk", type=int, default=8)
    ap.add_argument("--instances", type=int, default=0, help="override the instance count (profiling)")
    ap.add_argument("--tile-lanes", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--lanes-per-thread", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--job-points", type=int, default=12,
                    help="points of the job at which the per-cycle time is measured (0: skip the job leg)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--tune-kernels", default="",
                    help="comma-separated forms to autotune over (default: the library's choice for the "
                         "lane count: tile, grid, stream from 64 lanes, else layer, grid, cluster, flow)")
    ap.add_argument("--tune-log", default="")
    ap.add_argument("--no-verify", dest="verify", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

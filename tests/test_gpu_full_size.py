"""Parity at the workloads' full sizes, on sampled instances the oracle can follow.

* single-200k: 200k-op DAG, 1 instance, plain per-layer form and the grid form;
  and the whole configuration -- reset + 100,000 cycles -- in the CUDA-graph
  plain form, the cluster form and the FLOW form, every signal checked (the
  oracle runs alongside on the host);
* batch-1M: 1M ops, 4,096 instances with uneven cycle budgets, in the launch
  configuration the benchmark times (autotuned), five sampled instances
  (first, middle, last lane, shortest and longest budget) checked signal by signal;
  and the configuration's own budgets (uniform in [1k, 100k]) run for the
  first 2,000 cycles of the job: the shortest-budget instance (it finishes
  inside the run), one whose budget ends between 1k and 2k cycles and two
  still running, every signal;
* soc-5M: 5M ops, 256k registers, 64 register files (2 read, 1 write port
  each), 1,024 instances, reset + 2,000 cycles, two sampled instances, every
  signal and memory word.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def test_single_200k_plain_and_grid():
    nl = synth.generate(synth.spec_single())
    for kernel in ["layer", "grid"]:
        p = Pair(nl, 1, kernel=kernel, seed=1)
        p.step(1, reset=True)
        p.step(300)
        p.compare()
        p.close()


def test_single_200k_full_length():
    import threading

    import oracle
    import paper_2601_18140_gb300 as rt
    nl = synth.generate(synth.spec_single())
    xs = synth.xorshift_seeds(1, nl.n_inputs, 1)
    o = oracle.OracleSim(nl.to_bytes(), 1)
    oxs = xs.copy()

    def run_oracle():
        o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs)
        o.step(100_000, mode=oracle.STIM_XORSHIFT, xs=oxs)

    t = threading.Thread(target=run_oracle)    # the C oracle runs without the GIL
    t.start()
    d = rt.Design(nl.to_bytes())
    got = {}
    for kernel in ["layer_graph", "cluster", "flow"]:   # the plain form and the two one-instance forms
        s = rt.Sim(d, 1, kernel=kernel, xorshift_seed=xs)
        s.step(1, stimulus="xorshift", reset=True)
        s.step(100_000, stimulus="xorshift")
        got[kernel] = s.read()
        s.close()
    t.join()
    for kernel, g in got.items():
        assert np.array_equal(g, o.read()), kernel
    d.close()


def test_batch_1m_bench_configuration():
    nl = synth.generate(synth.spec_batch())
    n = 4096
    budgets = synth.cycle_budgets(5, n, 3, 12)
    # first / middle / last lane, and the instances with the shortest and longest budgets
    sample = sorted({0, n // 2, n - 1, int(np.argmin(budgets)), int(np.argmax(budgets))})
    p = Pair(nl, n, kernel="grid", seed=5, expected_cycles=budgets, oracle_instances=sample,
             threads=512, ctas_per_sm=2, lanes_per_thread=8, unroll=1)
    p.step(1, reset=True)
    p.sim.autotune(cycles_per_trial=1, kernels=["grid", "stream"])   # as the benchmark does
    p.step(budgets, threads=3)
    p.step(4, threads=3)
    p.compare()
    p.close()


def test_batch_1m_job_budgets_first_2000_cycles():
    nl = synth.generate(synth.spec_batch())
    n = 4096
    budgets = synth.cycle_budgets(5, n, 1000, 100_000)
    order = np.argsort(budgets, kind="stable")
    mid = [int(i) for i in order if 1000 < budgets[i] < 2000]
    assert mid, "no budget between 1k and 2k cycles"
    running = [int(i) for i in order[-2:]] + [int(order[n // 2])]
    sample = sorted({int(order[0]), mid[len(mid) // 2], *running})
    p = Pair(nl, n, kernel="grid", seed=5, expected_cycles=budgets, oracle_instances=sample,
             threads=224, ctas_per_sm=4, lanes_per_thread=8, unroll=1)
    p.step(1, reset=True, threads=len(sample))
    run = np.minimum(budgets, 2000).astype(np.uint32)
    done = np.zeros(n, np.uint32)
    for _ in range(4):   # four steps of up to 500 cycles: the live span shrinks as instances finish
        per = np.minimum(run - done, 500).astype(np.uint32)
        p.step(per, threads=len(sample))
        done += per
    assert np.array_equal(done, run)
    p.compare()
    p.close()


def test_soc_5m_with_memories():
    nl = synth.generate(synth.spec_soc())
    assert nl.n_mems == 64 and nl.n_wports == 64
    assert int((nl.op_code == synth.OP["MEMRD"]).sum()) == 128
    n = 1024
    p = Pair(nl, n, kernel="grid", seed=3, oracle_instances=[1, n - 2])
    p.step(1, reset=True, threads=2)
    for _ in range(4):   # 2,000 cycles, in four steps
        p.step(500, threads=2)
    p.compare()
    p.close()

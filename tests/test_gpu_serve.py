"""Serving on the GPU: jobs of three designs arrive over time, are admitted into
resident lane pools while others run (continuous batching), and each job's
result must be bit-identical to the same job run alone -- and to the oracle."""
import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300.serve import Job, build_server, latency_stats
from synth import DesignSpec

pytestmark = pytest.mark.gpu


def designs():
    return {
        "small": synth.generate(DesignSpec(n_ops=1500, n_regs=60, depth=8, n_inputs=4, seed=61,
                                           input_widths=(8, 16, 1, 64))),
        "mid": synth.generate(DesignSpec(n_ops=6000, n_regs=300, depth=20, n_inputs=8, seed=62)),
        "mem": synth.generate(DesignSpec(n_ops=3000, n_regs=100, depth=12, n_inputs=4, seed=63,
                                         input_widths=(8, 32, 5, 1), n_mems=4, mem_words=16)),
    }


def test_results_identical_alone_and_in_the_mix():
    nls = designs()
    srv = build_server({k: v.to_bytes() for k, v in nls.items()},
                       capacity={"small": 256, "mid": 128, "mem": 128}, quantum=37)
    rng = np.random.default_rng(7)
    names = list(nls)
    trace = [Job(k, names[k % 3], int(rng.integers(1, 41)), int(rng.integers(20, 300)),
                 seed=500 + k, arrival=0.004 * k) for k in range(24)]
    done = srv.run(trace)
    assert len(done) == 24 and srv.rounds > 3
    stats = latency_stats(done)
    assert stats["n"] == 24 and stats["p99_s"] >= stats["p50_s"] > 0
    # overlap: some job was admitted while another of its design was still running
    assert any(a.design == b.design and a.admitted < b.finished and b.admitted < a.finished
               for a in done for b in done if a.job_id < b.job_id)
    for job in done:
        nl = nls[job.design]
        xs = synth.xorshift_seeds(job.seed, nl.n_inputs, job.n_instances)
        alone = rt.Sim(srv.designs[job.design], job.n_instances, xorshift_seed=xs)
        alone.step(1, stimulus="xorshift", reset=True)
        alone.step(job.cycles, stimulus="xorshift")
        regs = np.arange(nl.reg_base, nl.reg_base + nl.n_regs)
        assert np.array_equal(alone.read(regs), job.result), job.job_id
        alone.close()
    for job in done[:3]:
        nl = nls[job.design]
        o = oracle.OracleSim(nl.to_bytes(), job.n_instances)
        oxs = synth.xorshift_seeds(job.seed, nl.n_inputs, job.n_instances)
        o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs)
        o.step(job.cycles, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=8)
        assert np.array_equal(o.read(np.arange(nl.reg_base, nl.reg_base + nl.n_regs)), job.result)


def test_reset_lanes_and_per_instance_reset():
    """A lane range returned to a fresh state and reset while neighbours keep running."""
    nl = designs()["mem"]
    d = rt.Design(nl.to_bytes())
    n = 128
    xs = synth.xorshift_seeds(9, nl.n_inputs, n)
    s = rt.Sim(d, n, xorshift_seed=xs)
    s.step(1, stimulus="xorshift", reset=True)
    s.step(40, stimulus="xorshift")
    before = s.read()
    new_seed = synth.xorshift_seeds(10, nl.n_inputs, 16)
    s.reset_lanes(32, 16, new_seed)
    rst = np.zeros(n, np.uint32)
    rst[32:48] = 1
    s.step(25, stimulus="xorshift", reset_per_instance=rst)
    after = s.read()
    ref = rt.Sim(d, 16, xorshift_seed=new_seed)
    ref.step(1, stimulus="xorshift", reset=True)
    ref.step(24, stimulus="xorshift")
    assert np.array_equal(after[:, 32:48], ref.read())
    cont = rt.Sim(d, n, xorshift_seed=xs)
    cont.step(1, stimulus="xorshift", reset=True)
    cont.step(65, stimulus="xorshift")
    keep = np.r_[0:32, 48:n]
    assert np.array_equal(after[:, keep], cont.read()[:, keep])
    for x in (s, ref, cont):
        x.close()
    d.close()

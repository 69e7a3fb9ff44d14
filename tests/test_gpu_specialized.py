"""Design-specialised form (Sec. 5.2 SU / TI on the GPU: the op list unrolled
into run-time-compiled straight-line code, one thread per instance): bit-exact
with the oracle, and its state is the data-driven kernels' state."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from synth import DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def design(seed, n_ops=700, n_mems=2):
    return synth.generate(DesignSpec(n_ops=n_ops, n_regs=50, depth=10, n_inputs=4, input_widths=(8, 32, 64, 1),
                                     seed=seed, n_mems=n_mems, mem_words=8))


def test_specialized_matches_oracle_with_switches():
    nl = design(51)
    n = 333
    rng = np.random.default_rng(51)
    budgets = rng.integers(0, 40, n).astype(np.uint32)
    p = Pair(nl, n, kernel="specialized", seed=51, expected_cycles=budgets)
    assert p.design.specialize() >= 0.0          # compiled once per design
    p.step(1, reset=True)
    p.step(17)
    p.compare()
    p.step(budgets)                               # uneven cycle counts
    p.compare()
    p.sim.configure(kernel="grid")                # the state is shared by every form
    p.step(5)
    p.sim.configure(kernel="specialized")
    p.step(9, stimulus="hold")
    vals = synth.stimulus_values(52, 6, nl.n_inputs, n)
    p.step(6, stimulus="buffer", values=vals)
    p.step(4, probes=[nl.reg_base, nl.op_base + 7, nl.n_signals - 1], probe_mode="last")
    p.compare()
    with pytest.raises(rt.RteaalError) as ei:
        p.sim.step(2, probes=[nl.reg_base], probe_mode="every")
    assert ei.value.code == rt.RTEAAL_E_UNSUPPORTED
    p.close()


def test_specialized_single_instance_and_per_instance_reset():
    nl = synth.generate(synth.spec_tiny(seed=3))
    p = Pair(nl, 1, kernel="specialized", seed=3)
    p.step(1, reset=True)
    p.step(2000)
    p.compare()
    p.close()
    nl = design(53, n_mems=0)
    d = rt.Design(nl.to_bytes())
    n = 64
    xs = synth.xorshift_seeds(53, nl.n_inputs, n)
    a = rt.Sim(d, n, kernel="specialized", xorshift_seed=xs)
    b = rt.Sim(d, n, kernel="layer", xorshift_seed=xs)
    rst = (np.arange(n) % 3).astype(np.uint32)   # 0, 1 or 2 leading reset cycles
    for s in (a, b):
        s.step(1, stimulus="xorshift", reset=True)
        s.step(12, stimulus="xorshift")
        s.step(7, stimulus="xorshift", reset_per_instance=rst)
    assert np.array_equal(a.read(), b.read())
    a.close()
    b.close()
    d.close()


def test_specialized_fused_design():
    nl = synth.generate(DesignSpec(n_ops=1500, n_regs=60, depth=12, n_inputs=4, seed=54,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7))
    d = rt.Design(nl.to_bytes(), fuse_mux_chains=True)
    assert d.info["n_fused"] > 0
    n = 96
    xs = synth.xorshift_seeds(54, nl.n_inputs, n)
    a = rt.Sim(d, n, kernel="specialized", xorshift_seed=xs)
    b = rt.Sim(d, n, kernel="grid", xorshift_seed=xs)
    for s in (a, b):
        s.step(1, stimulus="xorshift", reset=True)
        s.step(30, stimulus="xorshift")
    live = d.present_signals()
    assert np.array_equal(a.read(live), b.read(live))
    a.close()
    b.close()
    d.close()

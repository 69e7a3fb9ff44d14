"""Operator fusion of mux chains (App. B.1): the fused design evaluated on the
GPU equals the oracle run on the *unfused* netlist on every signal that still
exists; fused-away signals are refused."""
import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from synth import OP, DesignSpec
from tests.netlist_rules import fused_away

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", ["layer", "grid", "stream", "flow"])
def test_fused_mux_chains_match_unfused_oracle(kernel):
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=150, depth=16, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7, n_mems=2,
                                   mem_words=8))
    gone = fused_away(nl)
    assert len(gone) > 150
    d = rt.Design(nl.to_bytes(), fuse_mux_chains=True)
    assert d.info["n_fused"] == len(gone)
    assert d.info["n_lowered_ops"] == nl.n_ops - len(gone)
    n = 256
    xs = synth.xorshift_seeds(71, nl.n_inputs, n)
    s = rt.Sim(d, n, kernel=kernel, xorshift_seed=xs)
    s.step(1, stimulus="xorshift", reset=True)
    s.step(40, stimulus="xorshift")
    o = oracle.OracleSim(nl.to_bytes(), n)
    oxs = xs.copy()
    o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs)
    o.step(40, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=8)
    keep = np.array([x for x in range(nl.n_signals) if x not in gone])
    assert np.array_equal(d.present_signals(), keep)
    assert np.array_equal(s.read(keep), o.read(keep))
    assert np.array_equal(s.read_mem(), o.read_mem())
    with pytest.raises(rt.RteaalError):
        s.read([min(gone)])
    s.close()
    d.close()

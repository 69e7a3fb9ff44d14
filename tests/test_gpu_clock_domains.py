"""Multiple clock domains (Sec. 6.2): registers of slower domains load only on
their ticks.  The library lowers the domains to one clock (a hidden cycle
counter and hold muxes); every kernel form must match the oracle, which
implements the domain rule directly."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from synth import DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def multi_clock_design(seed=81):
    nl = synth.generate(DesignSpec(n_ops=900, n_regs=80, depth=12, n_inputs=4, seed=seed,
                                   input_widths=(8, 32, 1, 64), n_mems=2, mem_words=8))
    rng = np.random.default_rng(seed)
    nl.dom_period = np.array([1, 2, 4, 8, 32], np.uint32)
    nl.dom_phase = np.array([0, 1, 0, 5, 17], np.uint32)
    nl.reg_domain = rng.integers(0, 5, nl.n_regs).astype(np.uint8)
    return nl


@pytest.mark.parametrize("kernel", ["layer", "layer_graph", "tile", "grid", "stream", "specialized"])
def test_multi_clock_matches_oracle(kernel):
    nl = multi_clock_design()
    n = 200
    rng = np.random.default_rng(5)
    budgets = rng.integers(0, 50, n).astype(np.uint32)
    p = Pair(nl, n, kernel=kernel, seed=81, expected_cycles=budgets)
    assert p.design.info["n_regs"] == nl.n_regs           # the hidden counter is not a signal
    p.step(1, reset=True)
    p.step(37)
    p.compare()
    p.step(budgets)                                       # every instance at its own t
    p.compare()
    p.step(1, reset=True)                                 # a reset restarts the domains' phase
    p.step(21, probes=[nl.reg_base, nl.reg_base + 3, nl.op_base + 11],
           probe_mode="last")
    p.compare()
    p.close()


def test_multi_clock_activity_and_fusion():
    nl = multi_clock_design(82)
    n = 256
    for kw in [dict(activity=True), dict()]:
        p = Pair(nl, n, kernel="grid", seed=82, **kw)
        p.step(1, reset=True)
        p.step(60, stimulus="hold" if kw else "xorshift")
        p.compare()
        p.close()
    d = rt.Design(nl.to_bytes(), fuse_mux_chains=True)
    assert d.info["n_signals"] == nl.n_signals
    d.close()

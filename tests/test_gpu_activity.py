"""Activity-aware evaluation (App. B, skipping what did not change): results are
bit-identical to the oracle, and on an enable-gated modular design most
(op, lane-chunk) items are skipped."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def quiet(seed=6):
    return synth.generate_modular(synth.ModularSpec(n_modules=12, ops_per_module=1200, regs_per_module=80,
                                                    depth=14, seed=seed))


def test_quiet_design_matches_oracle_and_skips():
    nl = quiet()
    n = 384
    p = Pair(nl, n, kernel="grid", seed=6, activity=True)
    assert p.sim.info["activity"] == 1
    p.step(1, reset=True)                      # inputs take random per-instance values ...
    p.step(3)
    p.step(70, stimulus="hold")                # ... then hold: only enabled modules move
    p.compare()
    ev, sk = p.sim.activity()
    assert sk > 4 * ev                         # most items skipped
    p.step(45, stimulus="hold")
    p.compare()
    p.close()


@pytest.mark.parametrize("lanes_per_thread", [1, 2, 4, 8])
def test_random_design_uneven_budgets_and_writes(lanes_per_thread):
    """High-activity random design, per-instance budgets (the next step's first
    cycle re-evaluates everything), state writes and lane resets in between."""
    nl = synth.generate(synth.DesignSpec(n_ops=900, n_regs=60, depth=12, n_inputs=4, seed=7,
                                         input_widths=(8, 32, 1, 64), n_mems=2, mem_words=8))
    n = 300
    rng = np.random.default_rng(lanes_per_thread)
    budgets = rng.integers(0, 25, n).astype(np.uint32)
    p = Pair(nl, n, kernel="grid", seed=7, activity=True, lanes_per_thread=lanes_per_thread)
    p.step(1, reset=True)
    p.step(budgets)
    p.step(9, stimulus="hold")
    p.compare()
    # an external write: both sides get the same values
    regs = np.arange(nl.reg_base, nl.reg_base + 5)
    vals = (np.arange(5 * n, dtype=np.uint64).reshape(5, n) * np.uint64(0x9E3779B97F4A7C15))
    vals &= np.uint64(1)                     # fits every width
    p.sim.write(regs, vals)
    p.orc.vals[:, regs] = vals[:, p.sample].T
    p.step(6, stimulus="hold")
    p.step(budgets[::-1].copy())
    p.compare()
    p.close()


def test_activity_needs_the_grid_kernel():
    nl = quiet(8)
    d = rt.Design(nl.to_bytes())
    with pytest.raises(rt.RteaalError) as ei:
        rt.Sim(d, 128, kernel="tile", activity=True)
    assert ei.value.code == rt.RTEAAL_E_UNSUPPORTED
    s = rt.Sim(d, 128, activity=True)          # auto picks the grid kernel
    assert s.info["kernel"] == rt.KERNELS["grid"]
    with pytest.raises(rt.RteaalError):
        s.configure(kernel="stream")
    s.close()
    d.close()

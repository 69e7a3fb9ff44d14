"""Runtime behaviour on the GPU: reconfiguration, the autotuner, bounded waits."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from synth import DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def design(seed=12, n_mems=2):
    return synth.generate(DesignSpec(n_ops=800, n_regs=50, depth=12, n_inputs=4,
                                     input_widths=(8, 32, 64, 1), seed=seed, n_mems=n_mems,
                                     mem_words=8))


def test_configure_between_steps():
    nl = design()
    p = Pair(nl, 128, kernel="tile", seed=12)
    p.step(1, reset=True)
    with pytest.raises(rt.RteaalError) as ei:                 # no such compiled variant
        p.sim.configure(kernel="tile", tile_lanes=8, threads=1024, unroll=4)
    assert ei.value.code == rt.RTEAAL_E_UNSUPPORTED
    for cfg in [dict(kernel="tile", tile_lanes=8, threads=1024, unroll=1),
                dict(kernel="tile", tile_lanes=16, threads=512, unroll=2),
                dict(kernel="grid", threads=256, unroll=4),
                dict(kernel="layer", unroll=1),
                dict(kernel="tile", tile_lanes=64, threads=512, unroll=4),
                dict(kernel="layer_graph"),
                dict(kernel="stream")]:
        p.sim.configure(**cfg)
        p.step(7)
        p.compare()
    p.close()


def test_autotune_restores_state_exactly():
    nl = design(13)
    p = Pair(nl, 256, kernel="tile", seed=13)
    p.step(1, reset=True)
    p.step(5)
    before = p.sim.read()
    trials = p.sim.autotune(cycles_per_trial=2, kernels=["tile", "grid", "layer", "stream"])
    assert len(trials) >= 10
    assert all(t["ms"] > 0 for t in trials)
    assert np.array_equal(p.sim.read(), before)        # snapshot restored
    p.step(9)
    p.compare()
    p.close()


def test_grid_barrier_timeout_is_reported(monkeypatch):
    """Every grid-barrier wait is bounded: with one arrival withheld the kernel
    gives up after the limit, the step reports RTEAAL_E_TIMEOUT, and the
    device stays usable."""
    nl = design(14, n_mems=0)
    d = rt.Design(nl.to_bytes())
    monkeypatch.setenv("RTEAAL_TEST_WITHHOLD_ARRIVAL", "1")
    monkeypatch.setenv("RTEAAL_BARRIER_TIMEOUT_NS", "200000000")
    s = rt.Sim(d, 64, kernel="grid", threads=256)
    with pytest.raises(rt.RteaalError) as ei:
        s.step(3, stimulus="hold")
        s.sync()
    assert ei.value.code == rt.RTEAAL_E_TIMEOUT
    s.close()
    monkeypatch.delenv("RTEAAL_TEST_WITHHOLD_ARRIVAL")
    monkeypatch.delenv("RTEAAL_BARRIER_TIMEOUT_NS")
    p = Pair(nl, 64, kernel="grid", seed=14)
    p.step(1, reset=True)
    p.step(4)
    p.compare()
    p.close()
    d.close()


def test_design_free_refused_while_sims_live():
    nl = design(15)
    d = rt.Design(nl.to_bytes())
    s = rt.Sim(d, 2)
    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_design_free(d.handle)
    assert ei.value.code == rt.RTEAAL_E_BUSY
    s.close()
    d.close()


def test_footprint_matches_allocation():
    nl = design(16)
    d = rt.Design(nl.to_bytes())
    for n in [1, 100, 1000]:
        s = rt.Sim(d, n)
        assert s.info["device_bytes"] <= d.footprint(n)
        s.close()
    d.close()


def test_invalid_arguments_raise():
    nl = design(17)
    d = rt.Design(nl.to_bytes())
    with pytest.raises(rt.RteaalError):
        rt.Sim(d, 64, kernel="tile", tile_lanes=3)
    s = rt.Sim(d, 4)
    with pytest.raises(rt.RteaalError):
        s.read([nl.n_signals + 10])
    with pytest.raises(rt.RteaalError):
        s.read([0], inst_begin=3, n_inst=5)
    s.close()
    d.close()

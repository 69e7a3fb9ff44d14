"""The cluster form (thread-block clusters with the hardware cluster barrier
between layers) against the oracle: one instance (a one-lane tile, one lane
per thread) of a mid-size design over many cycles, every signal; several lane
tiles with uneven budgets (tiles retire at different cycles) and memories;
every cluster size the library accepts from 2 to 16 CTAs."""
import numpy as np
import pytest

import synth
from synth import DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("resident,cluster_ctas", [(-1, 0), (1, 4), (1, 8), (1, 16)])
def test_single_instance_many_cycles(resident, cluster_ctas):
    """One instance, 400 cycles, every signal and memory word; the state in
    global memory (resident = -1) or kept in the cluster's distributed shared
    memory (resident = 1) over clusters of 4, 8 and 16 CTAs."""
    nl = synth.generate(DesignSpec(n_ops=20_000, n_regs=2_000, depth=30, n_inputs=8, seed=61, n_mems=2,
                                   mem_words=16))
    p = Pair(nl, 1, kernel="cluster", seed=61, cluster_resident=resident, cluster_ctas=cluster_ctas)
    info = p.sim.info
    assert info["kernel"] == 7 and info["lanes_per_thread"] == 1 and info["cluster_ctas"] >= 2
    assert info["cluster_resident"] == (1 if resident == 1 else 0)
    if cluster_ctas:
        assert info["cluster_ctas"] == cluster_ctas
    p.step(1, reset=True)
    p.step(400)
    p.compare()
    probes = [0, nl.reg_base, nl.reg_base + 5, nl.op_base + 11, nl.n_signals - 1]
    p.step(9, probes=probes, probe_mode="every")
    p.compare()
    p.close()


def test_resident_lanes_uneven_budgets():
    """64 lanes kept in distributed shared memory: uneven budgets (lanes stop at
    their own counts inside one launch), then probes of the last cycle."""
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=200, depth=16, n_inputs=4, seed=63,
                                   input_widths=(8, 32, 64, 1), n_mems=1, mem_words=8))
    n = 64
    budgets = synth.cycle_budgets(63, n, 0, 50)
    p = Pair(nl, n, kernel="cluster", seed=63, expected_cycles=budgets, cluster_resident=1)
    assert p.sim.info["cluster_resident"] == 1
    p.step(1, reset=True)
    p.step(budgets)
    p.compare()
    p.step(13, probes=[nl.reg_base, nl.op_base + 3], probe_mode="last")
    p.compare()
    p.close()


@pytest.mark.parametrize("cluster_ctas,tile_lanes", [(16, 128), (8, 256), (2, 128)])
def test_tiles_uneven_budgets_and_memories(cluster_ctas, tile_lanes):
    nl = synth.generate(DesignSpec(n_ops=3000, n_regs=120, depth=12, n_inputs=4, seed=62,
                                   input_widths=(8, 32, 64, 1), n_mems=2, mem_words=8))
    n = 512
    budgets = synth.cycle_budgets(62, n, 0, 40)
    sample = sorted({0, 1, 127, 128, 255, 300, n - 1, int(np.argmax(budgets)), int(np.argmin(budgets))})
    p = Pair(nl, n, kernel="cluster", seed=62, expected_cycles=budgets, oracle_instances=sample,
             cluster_ctas=cluster_ctas, tile_lanes=tile_lanes)
    assert p.sim.info["cluster_ctas"] == cluster_ctas and p.sim.info["tile_lanes"] == tile_lanes
    p.step(1, reset=True)
    p.step(budgets)
    p.compare()
    p.step(budgets[::-1].copy())
    p.compare()
    p.close()

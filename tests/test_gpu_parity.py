"""Bit-exact parity of the CUDA path (through the C ABI) with the oracle."""
import numpy as np
import pytest

import synth
from synth import Builder, DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu

KERNELS = ["layer", "layer_graph", "tile", "grid", "stream", "cluster", "flow"]


def small_design(seed, n_ops=600, depth=10, n_regs=40, n_mems=0, inputs=(8, 32, 64, 1)):
    return synth.generate(DesignSpec(n_ops=n_ops, n_regs=n_regs, depth=depth, n_inputs=len(inputs),
                                     input_widths=inputs, seed=seed, n_mems=n_mems, mem_words=8))


def test_tiny_workload_single_instance_full_length():
    """2,000-op DAG + counter + LFSR, 1 instance: reset, then 10,000 cycles."""
    nl = synth.generate(synth.spec_tiny())
    p = Pair(nl, 1, kernel="layer")
    p.step(1, reset=True)
    p.step(10_000)
    p.compare()
    cnt = nl.reg_base + 64
    vals = p.sim.read([cnt, cnt + 1])
    assert int(vals[0, 0]) == 10_000                       # counter closed form
    assert int(vals[1, 0]) == 0x8786                        # LFSR after 10,000 steps (GF(2) pin)
    p.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_kernels_multi_instance_ragged(kernel):
    """100 instances: 4 tiles of 32 lanes, the last one ragged (4 real lanes)."""
    nl = synth.generate(synth.spec_tiny(seed=5))
    p = Pair(nl, 100, kernel=kernel, seed=5)
    p.step(1, reset=True)
    p.step(37)
    p.compare()
    p.step(0)
    p.step(5)
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_uneven_cycles_and_lane_order(kernel):
    nl = small_design(11, n_mems=3)
    n = 77
    rng = np.random.default_rng(0)
    budgets = rng.integers(0, 60, n).astype(np.uint32)
    p = Pair(nl, n, kernel=kernel, seed=11, expected_cycles=budgets)
    p.step(1, reset=True)
    p.step(budgets)
    p.compare()
    p.step(budgets[::-1].copy())
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel", ["layer", "tile", "grid"])
@pytest.mark.parametrize("tile_lanes,unroll,threads", [(64, 4, 256), (16, 1, 128), (8, 2, 512), (1, 2, 64)])
def test_tile_shapes(kernel, tile_lanes, unroll, threads):
    nl = small_design(3, n_mems=2)
    p = Pair(nl, 128, kernel=kernel, seed=3, tile_lanes=tile_lanes, unroll=unroll, threads=threads)
    p.step(1, reset=True)
    p.step(20)
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel,lanes", [(k, 0) for k in KERNELS] + [("grid", 8), ("tile", 8)])
def test_buffer_stimulus_and_probes(kernel, lanes):
    """Stimulus from a device buffer and held inputs; probes every cycle and at the
    last cycle (also at 8 lanes per thread, the benchmark's configuration)."""
    nl = small_design(21)
    n, c = 200, 12
    vals = synth.stimulus_values(21, c, nl.n_inputs, n)
    p = Pair(nl, n, kernel=kernel, seed=21, lanes_per_thread=lanes,
             tile_lanes=64 if (kernel == "tile" and lanes) else 0)
    p.step(1, reset=True, stimulus="hold")
    probes = [0, 1, nl.reg_base, nl.reg_base + 3, nl.op_base + 7, nl.n_signals - 1]
    p.step(c, stimulus="buffer", values=vals, probes=probes, probe_mode="every")
    p.compare()
    p.step(3, stimulus="hold", probes=probes, probe_mode="last")
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel,lanes", [("layer", 0), ("tile", 0), ("grid", 0), ("grid", 8), ("stream", 0),
                                          ("specialized", 0), ("cluster", 0), ("flow", 0)])
def test_wide_ops_and_memories(kernel, lanes):
    """Variadic folds (> 3 operands), long mux chains, two write ports per memory;
    the grid form also at 8 lanes per thread (the benchmark's configuration)."""
    b = Builder()
    ins = [b.input(w) for w in (64, 32, 8, 1, 1, 5)]
    m = b.mem(16, width=40)
    regs = [b.reg(w) for w in (64, 32, 40, 8)]
    ops = [b.op("ADD", 64, ins[0], ins[1], ins[2], regs[0], regs[1]),
           b.op("XOR", 32, ins[1], ins[2], regs[1], regs[3]),
           b.op("MUL", 64, ins[2], ins[5], regs[3], ins[2]),
           b.op("MUXCHAIN", 64, ins[3], ins[0], ins[4], regs[0], regs[3], ins[1], regs[2]),
           b.op("MUXCHAIN", 8, ins[4], regs[3], ins[2]),
           b.op("MEMRD", 40, ins[5], p0=m)]
    t = b.op("CAT", 64, ops[5], b.op("BITS", 24, ops[0], p0=30, p1=7), p0=24)
    b.write_port(m, ins[3], ins[2], ops[0])
    b.write_port(m, ins[4], ins[5], ops[2])
    b.connect(regs[0], t)
    b.connect(regs[1], ops[1])
    b.connect(regs[2], ops[3])
    b.connect(regs[3], ops[4])
    nl = b.build()
    p = Pair(nl, 200, kernel=kernel, seed=9, lanes_per_thread=lanes)
    p.step(1, reset=True)
    p.step(50)
    p.compare()
    p.close()


def test_register_chains_and_input_driven_registers():
    """Registers whose D is another register, an input or a constant."""
    b = Builder()
    x = b.input(16)
    r = [b.reg(16) for _ in range(4)]
    c = b.const(16, 0x1234)
    b.connect(r[0], x)
    b.connect(r[1], r[0])
    b.connect(r[2], r[1])
    b.connect(r[3], c)
    nl = b.build()
    for kernel in KERNELS:
        p = Pair(nl, 66, kernel=kernel, seed=2)
        p.step(1, reset=True)
        p.step(9)
        p.compare()
        p.close()


def test_no_inputs_no_registers():
    b = Builder()
    k = b.const(8, 7)
    b.op("ADD", 8, k, k)
    nl = b.build()
    p = Pair(nl, 3, kernel="layer")
    p.step(4)
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel", KERNELS + ["specialized"])
def test_designs_without_operations(kernel):
    """Degenerate designs: registers fed straight from inputs, constants and other
    registers (no combinational op at all: the edge reads copies the lowering
    inserts), and a design with nothing but one input."""
    b = Builder()
    i0 = b.input(8)
    i1 = b.input(64)
    k = b.const(16, 0xBEEF)
    r0 = b.reg(8, init=3)
    r1 = b.reg(64)
    r2 = b.reg(16)
    r3 = b.reg(8)
    b.connect(r0, i0)           # input -> register
    b.connect(r1, i1)
    b.connect(r2, k)            # constant -> register
    b.connect(r3, r0)           # register -> register (a 2-stage delay line)
    nl = b.build()
    assert nl.n_ops == 0
    n = 130
    p = Pair(nl, n, kernel=kernel, seed=9)
    p.step(1, reset=True)
    p.step(5)
    p.compare()
    rng = np.random.default_rng(9)
    budgets = rng.integers(0, 4, n).astype(np.uint32)
    p.step(budgets)
    p.compare()
    p.close()
    b = Builder()
    b.input(1)
    p = Pair(b.build(), 7 if kernel != "stream" else 128, kernel=kernel, seed=10)   # stream: 128-lane multiples
    p.step(3)
    p.compare()
    p.close()


def test_state_write_restore_checkpoint():
    """Run N cycles, snapshot, run M more; restore the snapshot and rerun M: same result."""
    nl = small_design(8, n_mems=2)
    p = Pair(nl, 64, kernel="tile", seed=8)
    p.step(1, reset=True)
    p.step(10)
    snap = p.sim.read()
    mem = p.sim.read_mem()
    xs = p.sim.read_stim_state()
    p.step(15)
    after = p.sim.read()
    p.sim.write(np.arange(nl.n_signals), snap)
    p.sim.write_mem(mem)
    p.sim.write_stim_state(xs)
    p.sim.step(15, stimulus="xorshift")
    assert np.array_equal(p.sim.read(), after)
    p.close()


def test_batch_invariance():
    """Instance i alone equals instance i inside a batch of 256 (tile form)."""
    nl = small_design(4)
    xs = synth.xorshift_seeds(4, nl.n_inputs, 256)
    import paper_2601_18140_gb300 as rt
    d = rt.Design(nl.to_bytes())
    big = rt.Sim(d, 256, kernel="tile", xorshift_seed=xs)
    big.step(1, reset=True, stimulus="xorshift")
    big.step(30, stimulus="xorshift")
    full = big.read()
    for i in [0, 77, 255]:
        one = rt.Sim(d, 1, kernel="layer", xorshift_seed=xs[:, i:i + 1])
        one.step(1, reset=True, stimulus="xorshift")
        one.step(30, stimulus="xorshift")
        assert np.array_equal(one.read()[:, 0], full[:, i])
        one.close()
    big.close()
    d.close()


@pytest.mark.parametrize("kernel", ["layer", "tile", "grid"])
@pytest.mark.parametrize("lanes_per_thread", [1, 2, 4, 8])
def test_lanes_per_thread(kernel, lanes_per_thread):
    """Every lanes-per-thread width (packed loads of 1, 2 or 4 lanes per row class)."""
    nl = small_design(31, n_mems=2)
    n = 200
    rng = np.random.default_rng(31)
    budgets = rng.integers(0, 25, n).astype(np.uint32)
    p = Pair(nl, n, kernel=kernel, seed=31, lanes_per_thread=lanes_per_thread,
             tile_lanes=32 if kernel == "tile" else 0)
    p.step(1, reset=True)
    p.step(20)
    p.step(budgets)
    p.compare()
    p.close()


@pytest.mark.parametrize("n", [128, 300, 1024, 1536])
def test_stream_chunks(n):
    """Stream form: chunks of 128 / 512 lanes, ragged tails, uneven budgets, memories, probes."""
    nl = small_design(41, n_ops=900, n_mems=3)
    rng = np.random.default_rng(n)
    budgets = rng.integers(0, 30, n).astype(np.uint32)
    p = Pair(nl, n, kernel="stream", seed=41, expected_cycles=budgets)
    p.step(1, reset=True)
    p.step(13, probes=[nl.reg_base, nl.op_base + 3, nl.n_signals - 1], probe_mode="every")
    p.step(budgets)
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel,lanes", [("layer", 0), ("tile", 0), ("grid", 0), ("grid", 8), ("stream", 0),
                                          ("flow", 0)])
def test_waveform_changes(kernel, lanes):
    """Device-side change records equal the changes derived from the oracle's trace."""
    from oracle.waveform import changes
    nl = small_design(51, n_mems=2)
    n = 130
    rng = np.random.default_rng(51)
    budgets = rng.integers(0, 17, n).astype(np.uint32)
    p = Pair(nl, n, kernel=kernel, seed=51, lanes_per_thread=lanes)
    p.step(1, reset=True)
    p.step(5)
    probes = [0, 3, nl.reg_base, nl.reg_base + 7, nl.op_base + 11, nl.op_base + 400, nl.n_signals - 1]
    before = p.orc.read(probes)
    recs, count = p.sim.step(budgets, stimulus="xorshift", probes=probes, probe_mode="changes")
    tr = p.orc.step(budgets, mode=1, xs=p.oxs, probes=probes, probe_cycles=int(budgets.max()), threads=8)
    exp = changes(before, tr, budgets)
    assert count == len(exp) == len(recs)
    got = np.array(sorted((int(r["cycle"]), int(r["probe"]), int(r["instance"]), int(r["value"]))
                          for r in recs), dtype=np.uint64).reshape(-1, 4)
    assert np.array_equal(got, exp)
    p.compare()
    recs2, count2 = p.sim.step(3, stimulus="xorshift", probes=probes, probe_mode="changes",
                               change_capacity=5)
    assert len(recs2) == min(5, count2)                       # overflow: count kept, records capped
    p.close()


def test_stream_many_items_per_warp():
    """Wide layers (15k ops each) over 512 lanes: every warp of the stream form
    has about a dozen items per layer, so its ring wraps and its slots are
    reused many times within a layer and across layers."""
    nl = synth.generate(DesignSpec(n_ops=60_000, n_regs=1000, depth=4, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 64, 1), n_mems=1, mem_words=8))
    n = 512
    budgets = synth.cycle_budgets(71, n, 5, 30)
    p = Pair(nl, n, kernel="stream", seed=71, expected_cycles=budgets,
             oracle_instances=[0, 129, 255, 256, 400, n - 1])
    p.step(1, reset=True)
    p.step(budgets)
    p.step(7)
    p.compare()
    p.close()


@pytest.mark.parametrize("kernel,lanes", [("grid", 8), ("grid", 4), ("tile", 8), ("layer", 4), ("grid", 2)])
def test_byte_results_packed_lanes(kernel, lanes):
    """Every opcode with a result of at most 8 bits over operands of every narrow
    class (the packed byte-lane path at 4 and 8 lanes per thread, the lane-by-lane
    path at 2), shift amounts and bit ranges on both sides of a byte, with uneven
    budgets so that partial lane masks are stored."""
    from tests.test_layer_form_emulated_host import byte_results_design
    nl = byte_results_design()
    n = 96
    budgets = synth.cycle_budgets(57, n, 5, 40)
    p = Pair(nl, n, kernel=kernel, seed=57, expected_cycles=budgets, lanes_per_thread=lanes)
    assert p.sim.info["lanes_per_thread"] == lanes
    p.step(1, reset=True)
    p.step(budgets)
    p.compare()
    p.step(13)
    p.compare()
    p.close()

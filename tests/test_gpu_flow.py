"""The FLOW form (no barrier between layers: every result also goes to a word
stamped with its cycle, and an item waits until the operands it reads carry
this cycle's stamp) against the oracle, every signal, memory word and stimulus
state: one, three and 32 instances; uneven budgets (frozen lanes never stamp);
wide rows (two stamped words each), memories and write ports, variadic ops
(operands from the side array; fused mux chains are in the fusion tests),
clock domains; probes; a reset between steps;
switching forms between steps (a stamp never repeats across launches); and a
wait that nothing satisfies, which must end in RTEAAL_E_TIMEOUT with the device
still usable."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from synth import Builder, DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def mixed_design(seed: int) -> synth.Netlist:
    return synth.generate(DesignSpec(n_ops=6000, n_regs=300, depth=24, n_inputs=6, seed=seed,
                                     input_widths=(8, 32, 1, 64, 16, 3), n_mems=2, mem_words=16,
                                     mem_write_ports=2))


@pytest.mark.parametrize("n,threads", [(1, 128), (3, 64), (32, 256)])
def test_flow_matches_oracle(n, threads):
    nl = mixed_design(81)
    p = Pair(nl, n, kernel="flow", seed=81, threads=threads)
    info = p.sim.info
    assert info["kernel"] == rt.KERNELS["flow"] and info["lanes_per_thread"] == 1
    assert info["threads"] == threads
    p.step(1, reset=True)
    p.step(150)
    p.compare()
    probes = [0, nl.reg_base, nl.reg_base + 7, nl.op_base + 5, nl.n_signals - 1]
    p.step(11, probes=probes, probe_mode="every")
    p.compare()
    p.step(1, reset=True)
    p.step(37)
    p.compare()
    p.close()


def test_flow_uneven_budgets():
    nl = mixed_design(82)
    n = 32
    budgets = synth.cycle_budgets(82, n, 0, 60)
    p = Pair(nl, n, kernel="flow", seed=82, expected_cycles=budgets)
    p.step(1, reset=True)
    p.step(budgets)
    p.compare()
    p.step(budgets[::-1].copy())
    p.compare()
    assert p.sim.info["last_span"] <= n
    p.close()


def test_flow_clock_domains_and_variadic_ops():
    b = Builder()
    ins = [b.input(w) for w in (64, 32, 8, 1, 1, 5)]
    m = b.mem(16, width=40)
    regs = [b.reg(w) for w in (64, 32, 40, 8)]
    ops = [b.op("ADD", 64, ins[0], ins[1], ins[2], regs[0], regs[1]),
           b.op("XOR", 32, ins[1], ins[2], regs[1], regs[3]),
           b.op("MUL", 64, ins[2], ins[5], regs[3], ins[2]),
           b.op("XORR", 1, regs[0]),
           b.op("MEMRD", 40, ins[5], p0=m)]
    t = b.op("CAT", 64, ops[4], b.op("BITS", 24, ops[0], p0=30, p1=7), p0=24)
    b.write_port(m, ins[3], ins[2], ops[0])
    b.write_port(m, ops[3], ins[5], ops[2])
    b.connect(regs[0], t)
    b.connect(regs[1], b.op("DSHR", 32, ops[1], ins[5]))
    b.connect(regs[2], b.op("MUX", 40, ins[4], ops[4], regs[2]))
    b.connect(regs[3], b.op("SUB", 8, ins[2], regs[3]))
    b.clock(regs[1], b.domain(4, 1))
    b.clock(regs[3], b.domain(2, 0))
    nl = b.build()
    p = Pair(nl, 5, kernel="flow", seed=84)
    p.step(1, reset=True)
    p.step(64)
    p.compare()
    p.close()


def test_flow_between_other_forms():
    """Steps alternate between forms on one sim: the FLOW stamps of a later
    launch never equal an earlier one's, so words left from earlier steps are
    never taken for this cycle's results."""
    nl = mixed_design(85)
    p = Pair(nl, 4, kernel="flow", seed=85)
    p.step(1, reset=True)
    for kernel, cycles in [("flow", 20), ("grid", 7), ("flow", 1), ("layer", 5), ("flow", 33), ("flow", 2)]:
        p.sim.configure(kernel=kernel)
        p.step(cycles)
        p.compare()
    p.close()


def test_flow_wait_timeout_is_reported(monkeypatch):
    """Every stamp wait is bounded: with items waiting for a stamp one ahead
    (a word nothing writes) the kernel gives up after the limit, the step
    reports RTEAAL_E_TIMEOUT, and the device stays usable."""
    nl = mixed_design(86)
    d = rt.Design(nl.to_bytes())
    monkeypatch.setenv("RTEAAL_TEST_FLOW_STAMP_SKEW", "1")
    monkeypatch.setenv("RTEAAL_BARRIER_TIMEOUT_NS", "200000000")
    s = rt.Sim(d, 2, kernel="flow")
    with pytest.raises(rt.RteaalError) as ei:
        s.step(3, stimulus="hold")
        s.sync()
    assert ei.value.code == rt.RTEAAL_E_TIMEOUT
    assert "FLOW" in str(ei.value)
    s.close()
    monkeypatch.delenv("RTEAAL_TEST_FLOW_STAMP_SKEW")
    monkeypatch.delenv("RTEAAL_BARRIER_TIMEOUT_NS")
    p = Pair(nl, 2, kernel="flow", seed=86)
    p.step(1, reset=True)
    p.step(9)
    p.compare()
    p.close()
    d.close()

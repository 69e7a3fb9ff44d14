"""The library's clock-domain lowering checked on the host (no GPU): the
one-clock netlist it builds (a hidden cycle counter, per slower domain an
enable, per register of such a domain a hold mux) is simulated by the oracle
as a plain one-clock design and must equal, signal for signal and memory word
for memory word, the oracle applying the domain rule (Sec. 6.2, "Multiple
Clock Domains") to the original netlist -- across uneven cycle counts and a
second reset that restarts every domain's phase."""
import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import Builder, DesignSpec


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()


def random_multi_clock(seed: int) -> synth.Netlist:
    nl = synth.generate(DesignSpec(n_ops=900, n_regs=80, depth=12, n_inputs=4, seed=seed,
                                   input_widths=(8, 32, 1, 64), n_mems=2, mem_words=8))
    rng = np.random.default_rng(seed)
    nl.dom_period = np.array([1, 2, 4, 8, 32, 1 << 31], np.uint32)
    nl.dom_phase = np.array([0, 1, 0, 5, 17, 3], np.uint32)
    nl.reg_domain = rng.integers(0, 6, nl.n_regs).astype(np.uint8)
    return nl


def counters() -> synth.Netlist:
    """One 16-bit counter per domain, including a domain of period 1 with a phase
    of 0 (ungated) and two domains sharing a period with different phases."""
    b = Builder()
    b.input(1)
    one = b.const(16, 1)
    for period, phase in [(1, 0), (2, 1), (4, 0), (4, 3), (16, 9)]:
        r = b.reg(16)
        b.connect(r, b.op("ADD", 16, r, one))
        b.clock(r, b.domain(period, phase))
    return b.build()


def run_both(nl: synth.Netlist, n: int, seed: int):
    one, user2x = rt.rteaal_design_single_clock(nl.to_bytes(), nl.n_signals)
    flat = synth.Netlist.from_bytes(one)
    assert flat.n_domains == 0 and flat.n_inputs == nl.n_inputs
    assert flat.n_regs == nl.n_regs + 1                     # the hidden cycle counter
    native = oracle.OracleSim(nl.to_bytes(), n)
    lowered = oracle.OracleSim(one, n)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n)
    xa, xb = xs.copy(), xs.copy()
    rng = np.random.default_rng(seed)
    mem = slice(0, native.mem_total)

    def step(cycles, reset=False):
        native.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xa)
        lowered.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xb)
        assert np.array_equal(native.vals, lowered.vals[:, user2x])
        assert np.array_equal(native.mems[:, mem], lowered.mems[:, mem])

    step(1, reset=True)
    step(37)
    step(rng.integers(0, 70, n).astype(np.uint32))          # every instance at its own t
    step(1, reset=True)                                      # a reset restarts the phases
    step(45)


def test_counters_per_domain():
    nl = counters()
    run_both(nl, 3, 1)
    # the closed form as well: after reset + 45 cycles a counter of domain (p, f)
    # holds #{t < 45 : (t + f) mod p == 0}
    sim = oracle.OracleSim(rt.rteaal_design_single_clock(nl.to_bytes(), nl.n_signals)[0], 1)
    sim.step(1, reset=True)
    sim.step(45)
    for r, (p, f) in enumerate([(1, 0), (2, 1), (4, 0), (4, 3), (16, 9)]):
        assert int(sim.vals[0, nl.reg_base + r]) == sum((t + f) % p == 0 for t in range(45))


@pytest.mark.parametrize("seed", [81, 82])
def test_random_designs_with_memories(seed):
    run_both(random_multi_clock(seed), 16, seed)


def test_one_clock_netlists_pass_through_unchanged():
    nl = synth.generate(synth.spec_tiny(0))
    one, user2x = rt.rteaal_design_single_clock(nl.to_bytes(), nl.n_signals)
    assert one == nl.to_bytes() and np.array_equal(user2x, np.arange(nl.n_signals))
    b = Builder()
    i0 = b.input(8)
    r = b.reg(8)
    b.connect(r, b.op("ADD", 8, r, i0))
    b.clock(r, b.domain(1, 0))                               # every domain of period 1: no counter
    nl = b.build()
    one, _ = rt.rteaal_design_single_clock(nl.to_bytes(), nl.n_signals)
    assert synth.Netlist.from_bytes(one).n_regs == 1

"""The whole lowering checked on the host (no GPU): the descriptors the kernels
execute -- ctl words (opcode, arity, width, parameters), operand row
references and side-array operand lists, the order of the rows, the copies the
clock edge reads, fused mux chains, the register and write-port tables, the
clock-domain counter and hold muxes -- are decoded back into a netlist
(rteaal_design_lowered_netlist), and the oracle simulating that netlist must
give every surviving signal and every memory word the value the oracle gives
them on the original netlist, over reset, uneven cycle counts and a second
reset."""
import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import Builder, DesignSpec

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()


def roundtrip(nl: synth.Netlist, fuse: bool = False, n: int = 12, seed: int = 1) -> np.ndarray:
    low, user2sig = rt.rteaal_design_lowered_netlist(nl.to_bytes(), nl.n_signals, fuse_mux_chains=fuse)
    kept = user2sig != NONE
    native = oracle.OracleSim(nl.to_bytes(), n)
    lowered = oracle.OracleSim(low, n)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n)
    xa, xb = xs.copy(), xs.copy()
    rng = np.random.default_rng(seed)

    def step(cycles, reset=False):
        native.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xa)
        lowered.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xb)
        assert np.array_equal(native.vals[:, kept], lowered.vals[:, user2sig[kept]])
        assert np.array_equal(native.mems[:, :native.mem_total], lowered.mems[:, :native.mem_total])

    step(1, reset=True)
    step(30)
    step(rng.integers(0, 40, n).astype(np.uint32))
    step(1, reset=True)
    step(17)
    return user2sig


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_designs_with_memories(seed):
    nl = synth.generate(DesignSpec(n_ops=2500, n_regs=150, depth=14, n_inputs=4, seed=seed,
                                   input_widths=(8, 32, 1, 64), n_mems=2 + seed, mem_words=8,
                                   mem_write_ports=1 + seed % 2))
    roundtrip(nl, seed=seed)


def test_counter_lfsr_design():
    roundtrip(synth.generate(synth.spec_tiny(0)), n=4)


@pytest.mark.parametrize("fuse", [False, True])
def test_mux_chains(fuse):
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=150, depth=16, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7, n_mems=2, mem_words=8))
    user2sig = roundtrip(nl, fuse)
    assert ((user2sig == NONE).sum() > 150) == fuse          # fused muxes have no row


def test_fusion_keeps_a_narrower_inner_mux():
    """A mux whose false operand is a narrower mux must not absorb it: the inner
    mask (8 bits here) would be lost under the head's (16 bits)."""
    b = Builder()
    s0, s1 = b.input(1), b.input(1)
    a, c, d = b.input(16), b.input(16), b.input(16)
    inner = b.op("MUX", 8, s1, c, d)
    head = b.op("MUX", 16, s0, a, inner)
    ok = b.op("MUX", 16, s1, c, d)                             # an equal-width chain is fused
    head2 = b.op("MUX", 16, s0, a, ok)
    r = b.reg(16)
    b.connect(r, b.op("XOR", 16, head, head2))
    nl = b.build()
    assert rt.rteaal_design_lower(nl.to_bytes(), fuse_mux_chains=True)[0]["n_fused"] == 1
    user2sig = roundtrip(nl, fuse=True, n=64)
    assert user2sig[b.sid(inner)] != NONE and user2sig[b.sid(ok)] == NONE


def test_wide_ops_and_memories():
    """Variadic folds (> 3 operands: side-array operand lists), user-written
    MUXCHAINs, MEMRD, CAT / BITS parameters, two write ports on one memory."""
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
    roundtrip(b.build(), n=16)


def test_clock_domains():
    nl = synth.generate(DesignSpec(n_ops=900, n_regs=80, depth=12, n_inputs=4, seed=81,
                                   input_widths=(8, 32, 1, 64), n_mems=2, mem_words=8))
    rng = np.random.default_rng(81)
    nl.dom_period = np.array([1, 2, 4, 8, 32], np.uint32)
    nl.dom_phase = np.array([0, 1, 0, 5, 17], np.uint32)
    nl.reg_domain = rng.integers(0, 5, nl.n_regs).astype(np.uint8)
    roundtrip(nl, n=8)
    roundtrip(nl, fuse=True, n=8)


def test_edge_copies_and_degenerate_designs():
    b = Builder()
    i0 = b.input(8)
    i1 = b.input(64)
    k = b.const(16, 0xBEEF)
    m = b.mem(4, 8)
    r0, r1, r2, r3 = b.reg(8, init=3), b.reg(64), b.reg(16), b.reg(8)
    b.connect(r0, i0)
    b.connect(r1, i1)
    b.connect(r2, k)
    b.connect(r3, r0)
    b.write_port(m, b.input(1), i0, r3)          # a write port fed by pool signals only
    roundtrip(b.build(), n=5)
    b = Builder()
    b.input(1)
    roundtrip(b.build(), n=3)


@pytest.mark.parametrize("fuse", [False, True])
def test_compact_layout(fuse):
    """Every row is stored at its width class (1, 2, 4 or 8 bytes per lane for
    widths up to 8, 16, 32, 64); the class-3 rows come first, then 2, 1, 0; inside
    a class the rows follow their ids (pool rows before op rows) with no gap, so
    the rows tile [0, state bytes per lane) exactly."""
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=150, depth=16, n_inputs=4, seed=72,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7, n_mems=2, mem_words=8))
    low, _ = rt.rteaal_design_lowered_netlist(nl.to_bytes(), nl.n_signals, fuse_mux_chains=fuse)
    x = synth.Netlist.from_bytes(low)
    refs = rt.rteaal_design_rows(nl.to_bytes(), x.n_signals, fuse_mux_chains=fuse).astype(np.int64)
    k, off = refs >> 30, refs & ((1 << 30) - 1)
    w = x.signal_widths().astype(np.int64)
    assert np.array_equal(k, np.select([w <= 8, w <= 16, w <= 32], [0, 1, 2], 3))
    size = np.int64(1) << k
    end = 0
    for cls in (3, 2, 1, 0):
        ids = np.flatnonzero(k == cls)                       # in id order
        assert np.array_equal(off[ids], end + size[ids].cumsum() - size[ids])
        end += int(size[ids].sum())
    info, _ = rt.rteaal_design_lower(nl.to_bytes(), fuse_mux_chains=fuse)
    assert end == info["state_bytes_per_lane"]


@pytest.mark.parametrize("fuse", [False, True])
def test_flow_tables(fuse):
    """The FLOW form's tables against the compact layout: every op's operand
    rows are its operands' ranks in layout order (class 3 first, then by
    offset), flagged exactly when the operand is an op result (written in the
    cycle, so its stamp is waited for); absent operands are 0; extended ops list
    their operand rows in the side array in O order; the output row and
    reference are the op's own; the pool lists inputs, registers and constants
    with their rows."""
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=150, depth=16, n_inputs=4, seed=73,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7, n_mems=2, mem_words=8))
    low, _ = rt.rteaal_design_lowered_netlist(nl.to_bytes(), nl.n_signals, fuse_mux_chains=fuse)
    x = synth.Netlist.from_bytes(low)
    refs = rt.rteaal_design_rows(nl.to_bytes(), x.n_signals, fuse_mux_chains=fuse).astype(np.int64)
    op, ext, pool = rt.rteaal_design_flow_tables(nl.to_bytes(), fuse_mux_chains=fuse)
    k, off = refs >> 30, refs & ((1 << 30) - 1)
    order = np.lexsort((off, -k))                  # layout order: class 3 first, then by offset
    row = np.empty(x.n_signals, np.int64)
    row[order] = np.arange(x.n_signals)
    check = 1 << 31

    def want(sig: int) -> int:
        return int(row[sig]) | (check if sig >= x.op_base else 0)

    assert op.shape == (x.n_ops, 8)
    n_ext = 0
    for i in range(x.n_ops):
        q = [int(v) for v in op[i]]
        args = [int(a) for a in x.op_args(i)]
        assert q[3] == row[x.op_base + i] and q[5] == refs[x.op_base + i]
        assert (q[4] >> 8) & 127 == x.op_width[i]
        if len(args) <= 3:
            assert q[:3] == [want(a) for a in args] + [0] * (3 - len(args)), i
        else:
            n_ext += 1
            assert q[:3] == [0, 0, 0]
            assert [int(v) for v in ext[q[6]:q[6] + q[7]]] == [want(a) for a in args], i
    assert (n_ext > 0) == fuse
    sigs = list(range(x.n_inputs)) + list(range(x.reg_base, x.reg_base + x.n_regs)) + \
        list(range(x.const_base, x.const_base + x.n_consts))
    assert pool.tolist() == [[int(refs[s]), int(row[s])] for s in sigs]

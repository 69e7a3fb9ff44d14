"""Oracle pins by brute force and by the paper's cascade (CPU only).

* every input assignment of tiny random circuits (<= 16 input bits): oracle.c
  against the pure-Python evaluator;
* the Einsum cascade of Sec. 4 (levels, explicit identity operations, O-order
  reduce, populate for selects) against oracle.c on random circuits that use
  every opcode, registers and memories;
* invariants the paper states: operations inside a layer are independent
  (permuting them changes nothing, Sec. 4.1), identity operations change no
  value (Sec. 4.3), and instances are independent (batch invariance).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.cascade import CascadeSim, levelize
from oracle.pyeval import PySim
from synth import OP, DesignSpec, Netlist

ALL_CLASSES = {"logic": 30, "addsub": 15, "mul": 5, "shift": 15, "compare": 10, "mux": 25}


def tiny(seed, n_ops=24, depth=4, n_regs=3, input_widths=(8, 8), n_mems=0, widths=None):
    spec = DesignSpec(n_ops=n_ops, n_regs=n_regs, depth=depth, n_inputs=len(input_widths),
                      n_consts=4, seed=seed, input_widths=input_widths, n_mems=n_mems,
                      mem_words=4, widths=widths or {1: 0.3, 4: 0.2, 8: 0.2, 16: 0.1, 32: 0.1, 64: 0.1})
    return synth.generate(spec)


@pytest.mark.parametrize("seed", [101, 202])
def test_bruteforce_all_16bit_inputs(seed):
    nl = tiny(seed)
    n = 1 << 16
    buf = np.stack([np.arange(n) & 255, np.arange(n) >> 8]).astype(np.uint64).reshape(1, 2, n)
    sim = oracle.OracleSim(nl.to_bytes(), n)
    sim.step(1, reset=True)
    sim.step(1, mode=oracle.STIM_BUFFER, buf=buf)
    got = sim.vals
    ps = PySim(nl)
    ps.cycle([0, 0], reset=True)
    base = list(ps.v)
    for i in range(n):
        ps.v = list(base)
        ps.cycle([i & 255, i >> 8])
        assert [int(x) for x in got[i]] == ps.v, i


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_bruteforce_12bit_inputs_multicycle(seed):
    """Every 12-bit input assignment held for 3 cycles after reset, registers live."""
    nl = tiny(seed, n_ops=30, depth=5, n_regs=6, input_widths=(4, 8))
    n = 1 << 12
    vals = np.stack([np.arange(n) & 15, np.arange(n) >> 4]).astype(np.uint64)
    buf = np.broadcast_to(vals, (3, 2, n)).copy()
    sim = oracle.OracleSim(nl.to_bytes(), n)
    sim.step(1, reset=True)
    sim.step(3, mode=oracle.STIM_BUFFER, buf=buf)
    ps0 = PySim(nl)
    ps0.cycle([0, 0], reset=True)
    base = list(ps0.v)
    for i in range(0, n, 3):
        ps = PySim(nl)
        ps.v = list(base)
        for _ in range(3):
            ps.cycle([i & 15, i >> 4])
        assert [int(x) for x in sim.vals[i]] == ps.v, i


@pytest.mark.parametrize("seed", [19, 25])     # seeds whose write ports write and reads vary
def test_bruteforce_memories_multicycle(seed):
    """Every 12-bit input assignment held for 4 cycles after reset with two
    register files (two read ports each, one or two write ports): values and
    every memory word against the pure-Python evaluator, so that a write is seen
    by the reads of the next cycle and not of its own."""
    nl = synth.generate(DesignSpec(n_ops=40, n_regs=6, depth=5, n_inputs=2, n_consts=4, seed=seed,
                                   input_widths=(4, 8), n_mems=2, mem_words=4, mem_read_ports=2,
                                   mem_write_ports=1 + seed % 2,
                                   widths={1: 0.3, 4: 0.2, 8: 0.2, 16: 0.1, 32: 0.1, 64: 0.1}))
    assert nl.n_mems == 2 and nl.n_wports >= 2
    n = 1 << 12
    vals = np.stack([np.arange(n) & 15, np.arange(n) >> 4]).astype(np.uint64)
    buf = np.broadcast_to(vals, (4, 2, n)).copy()
    sim = oracle.OracleSim(nl.to_bytes(), n)
    sim.step(1, reset=True)
    sim.step(4, mode=oracle.STIM_BUFFER, buf=buf)
    assert (nl.op_code == OP["MEMRD"]).sum() == 4
    assert (sim.mems != 0).mean() > 0.2                       # the write ports do write
    mr = np.flatnonzero(nl.op_code == OP["MEMRD"]) + nl.op_base
    assert max(np.unique(sim.vals[:, x]).size for x in mr) > 1  # and the reads see it
    for i in range(0, n, 5):
        ps = PySim(nl)
        ps.cycle([0, 0], reset=True)
        for _ in range(4):
            ps.cycle([i & 15, i >> 4])
        assert [int(x) for x in sim.vals[i]] == ps.v, i
        assert [int(x) for x in sim.mems[i, :sum(len(m) for m in ps.mem)]] == [w for m in ps.mem for w in m], i


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_cascade_matches_oracle(seed):
    nl = tiny(seed, n_ops=80, depth=6, n_regs=10, input_widths=(8, 16, 1, 64), n_mems=2)
    n_inst = 3
    cs = [CascadeSim(nl) for _ in range(n_inst)]
    assert cs[0].n_identity > 0                                 # identities are exercised
    sim = oracle.OracleSim(nl.to_bytes(), n_inst)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n_inst)
    xs_c = xs.copy()
    sim.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    ins = _xorshift_inputs(xs_c, 1)
    for i in range(n_inst):
        cs[i].cycle(ins[0][:, i], reset=True)
    for c in range(25):
        sim.step(1, mode=oracle.STIM_XORSHIFT, xs=xs)
        ins = _xorshift_inputs(xs_c, 1)
        for i in range(n_inst):
            cs[i].cycle(ins[0][:, i])
            assert [int(x) for x in sim.vals[i]] == cs[i].v, (c, i)
            assert [int(x) for x in sim.mems[i, : sim.mem_total]] == sum(cs[i].mem, [])


def _xorshift_inputs(xs, n):
    """Stimulus values drawn the way the testbench draws them (in place on xs)."""
    out = []
    M = (1 << 64) - 1
    for _ in range(n):
        vals = np.zeros_like(xs)
        for j in range(xs.shape[0]):
            for i in range(xs.shape[1]):
                x = int(xs[j, i])
                x ^= (x << 13) & M
                x ^= x >> 7
                x ^= (x << 17) & M
                xs[j, i] = x
                vals[j, i] = x
        out.append(vals)
    return out


def test_cascade_on_the_tiny_workload_design():
    nl = synth.generate(synth.spec_tiny())
    cs = CascadeSim(nl)
    assert cs.I == max(levelize(nl))
    sim = oracle.OracleSim(nl.to_bytes(), 1)
    xs = synth.xorshift_seeds(0, nl.n_inputs, 1)
    xs_c = xs.copy()
    sim.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    cs.cycle(_xorshift_inputs(xs_c, 1)[0][:, 0], reset=True)
    for _ in range(3):
        sim.step(1, mode=oracle.STIM_XORSHIFT, xs=xs)
        cs.cycle(_xorshift_inputs(xs_c, 1)[0][:, 0])
    assert [int(x) for x in sim.vals[0]] == cs.v


# ---------------------------------------------------------------- invariants
def permute_within_levels(nl: Netlist, seed: int) -> tuple[Netlist, np.ndarray]:
    """Reorder ops by (level, random key); returns the netlist and old->new signal map."""
    lvl = np.array(levelize(nl))
    rng = np.random.default_rng(seed)
    order = np.lexsort((rng.random(nl.n_ops), lvl[nl.op_base:]))   # new position -> old op
    remap = np.arange(nl.n_signals)
    remap[nl.op_base + order] = nl.op_base + np.arange(nl.n_ops)
    args = []
    argoff = [0]
    for k in order:
        args.extend(int(remap[a]) for a in nl.op_args(int(k)))
        argoff.append(len(args))
    out = Netlist(nl.input_width, nl.reg_width, remap[nl.reg_d].astype(np.uint32), nl.reg_init,
                  nl.const_width, nl.const_value, nl.op_code[order], nl.op_width[order],
                  nl.op_p0[order], nl.op_p1[order], np.array(argoff, np.uint32),
                  np.array(args, np.uint32), nl.mem_words, nl.mem_width,
                  np.concatenate([nl.wport[:, :1], remap[nl.wport[:, 1:]]], axis=1).astype(np.uint32))
    return out, remap


def insert_identities(nl: Netlist) -> tuple[Netlist, np.ndarray]:
    """Route every op operand through an explicit COPY op placed just before its consumer."""
    n_new = nl.n_ops + int(nl.args.size)
    new_base = nl.op_base
    remap = np.arange(nl.n_signals)
    code, width, p0, p1, args, argoff = [], [], [], [], [], [0]
    sw = nl.signal_widths()
    pos = 0
    for k in range(nl.n_ops):
        ops_args = []
        for a in nl.op_args(k):
            a2 = int(remap[a]) if a >= nl.op_base else int(a)
            code.append(OP["COPY"]); width.append(int(sw[a])); p0.append(0); p1.append(0)
            args.append(a2); argoff.append(len(args))
            ops_args.append(new_base + pos)
            pos += 1
        code.append(int(nl.op_code[k])); width.append(int(nl.op_width[k]))
        p0.append(int(nl.op_p0[k])); p1.append(int(nl.op_p1[k]))
        args.extend(ops_args); argoff.append(len(args))
        remap[nl.op_base + k] = new_base + pos
        pos += 1
    assert pos == n_new
    out = Netlist(nl.input_width, nl.reg_width, remap[nl.reg_d].astype(np.uint32), nl.reg_init,
                  nl.const_width, nl.const_value, np.array(code, np.uint8),
                  np.array(width, np.uint8), np.array(p0, np.uint8), np.array(p1, np.uint8),
                  np.array(argoff, np.uint32), np.array(args, np.uint32), nl.mem_words,
                  nl.mem_width,
                  np.concatenate([nl.wport[:, :1], remap[nl.wport[:, 1:]]], axis=1).astype(np.uint32))
    return out, remap


def _run(nl, n_inst, cycles, seed):
    sim = oracle.OracleSim(nl.to_bytes(), n_inst)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n_inst)
    sim.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    sim.step(cycles, mode=oracle.STIM_XORSHIFT, xs=xs)
    return sim


@pytest.mark.parametrize("seed", [5, 6])
def test_permuting_ops_within_a_layer(seed):
    nl = tiny(seed, n_ops=300, depth=8, n_regs=20, input_widths=(8, 32, 64), n_mems=2)
    pn, remap = permute_within_levels(nl, seed)
    assert not np.array_equal(pn.op_code, nl.op_code)
    a = _run(nl, 4, 40, seed)
    b = _run(pn, 4, 40, seed)
    assert np.array_equal(a.vals, b.vals[:, remap])
    assert np.array_equal(a.mems, b.mems)


def test_identity_operations_change_nothing():
    nl = tiny(3, n_ops=200, depth=8, n_regs=20, input_widths=(8, 32, 64), n_mems=1)
    inl, remap = insert_identities(nl)
    a = _run(nl, 4, 40, 3)
    b = _run(inl, 4, 40, 3)
    assert np.array_equal(a.vals, b.vals[:, remap])


def test_batch_invariance_and_threads():
    nl = tiny(4, n_ops=300, depth=8, n_regs=20, input_widths=(8, 32, 64))
    n = 16
    xs = synth.xorshift_seeds(9, nl.n_inputs, n)
    cyc = np.arange(n, dtype=np.uint32) * 3 + 1
    full = oracle.OracleSim(nl.to_bytes(), n)
    x1 = xs.copy()
    full.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=x1)
    full.step(cyc, mode=oracle.STIM_XORSHIFT, xs=x1, threads=4)
    for i in [0, 5, 15]:
        one = oracle.OracleSim(nl.to_bytes(), 1)
        x2 = xs[:, i:i + 1].copy()
        one.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=x2)
        one.step(int(cyc[i]), mode=oracle.STIM_XORSHIFT, xs=x2)
        assert np.array_equal(one.vals[0], full.vals[i])
        assert np.array_equal(x2[:, 0], x1[:, i])


def test_format_errors_rejected():
    nl = tiny(1)
    b = bytearray(nl.to_bytes())
    with pytest.raises(ValueError):
        oracle.OracleSim(bytes(b[:-1]), 1)
    bad = Netlist.from_bytes(bytes(b))
    bad.args[0] = bad.n_signals + 5                  # operand beyond the signal space
    with pytest.raises(ValueError):
        oracle.OracleSim(bad.to_bytes(), 1)

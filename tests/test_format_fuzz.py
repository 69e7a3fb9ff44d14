"""Malformed netlists on the host: seeded corruptions of valid RTLN netlists
(flipped bytes, header counts set to edge values, truncation, trailing bytes,
corrupted operand ids) never crash either parser, the library reports every
rejection as E_FORMAT, and the library's parser (with its lowering) and the
oracle's independent one accept exactly the same inputs; an accepted one-clock
netlist is lowered as the levelisation restated from it predicts, and the
oracle simulates it as the pure-Python evaluator and the Einsum cascade do; and
every accepted netlist's lowering, decoded back into a netlist, simulates like
it (with and without operator fusion); the other host-only calls accept and
refuse the same inputs, never crashing."""
import struct

import numpy as np

import oracle
import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import Builder, DesignSpec
from oracle.cascade import CascadeSim
from oracle.pyeval import PySim
from tests.test_lowering_host import check


def _bases() -> list[bytes]:
    out = [synth.generate(DesignSpec(n_ops=60, n_regs=5, depth=4, seed=s, n_mems=s % 2, mem_words=4)).to_bytes()
           for s in range(3)]
    b = Builder()
    i0 = b.input(8)
    r = b.reg(8)
    b.connect(r, b.op("ADD", 8, r, i0))
    b.clock(r, b.domain(4, 1))
    out.append(b.build().to_bytes())
    return out


def _corrupt(b: bytearray, rng) -> bytes:
    kind = rng.integers(0, 4)
    if kind == 0:                                   # flipped bytes
        for _ in range(rng.integers(1, 6)):
            b[rng.integers(0, len(b))] = rng.integers(0, 256)
    elif kind == 1:                                 # a header count set to an edge value
        i = rng.integers(2, 10)
        v = int(rng.choice([0, 1, 2, 255, 65535, 2**31, 2**32 - 1, rng.integers(0, 1000)]))
        b[4 * i:4 * i + 4] = struct.pack("<I", v)
    elif kind == 2:                                 # truncated or extended
        b = b[:rng.integers(0, len(b))] if rng.random() < 0.5 else b + bytes(int(rng.integers(1, 64)))
    else:                                           # a u32 of the body (ids, offsets, sizes)
        j = int(rng.integers(40, max(41, len(b) - 4))) & ~3
        b[j:j + 4] = struct.pack("<I", int(rng.choice([0xFFFFFFFF, 0x7FFFFFFF, rng.integers(0, 5000)])))
    return bytes(b)


def _same_as_pyeval(b: bytes, nl: synth.Netlist, rng, n_inst: int = 2, cycles: int = 4):
    ni = nl.n_inputs
    vals = rng.integers(0, 2**63, size=(cycles, ni, n_inst), dtype=np.uint64)
    sim = oracle.OracleSim(b, n_inst)
    sim.step(1, reset=True)
    sim.step(cycles, mode=oracle.STIM_BUFFER, buf=vals)
    for i in range(n_inst):
        ps = PySim(nl)
        ps.cycle([0] * ni, reset=True)
        for c in range(cycles):
            ps.cycle([int(x) for x in vals[c, :, i]])
        assert [int(x) for x in sim.vals[i]] == ps.v
    cs = CascadeSim(nl)
    cs.cycle(np.zeros(ni, np.uint64), reset=True)
    for c in range(cycles):
        cs.cycle(vals[c, :, 0])
    assert [int(x) for x in sim.vals[0]] == cs.v


def _lowering_simulates_alike(b: bytes, nl: synth.Netlist, fuse: bool, seed: int, n_inst: int = 2):
    low, user2sig = rt.rteaal_design_lowered_netlist(b, nl.n_signals, fuse)
    keep = user2sig != 0xFFFFFFFF
    native, lowered = oracle.OracleSim(b, n_inst), oracle.OracleSim(low, n_inst)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n_inst)
    xa, xb = xs.copy(), xs.copy()
    for cycles, reset in [(1, True), (5, False), (1, True), (3, False)]:
        native.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xa)
        lowered.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xb)
        assert np.array_equal(native.vals[:, keep], lowered.vals[:, user2sig[keep]])
        assert np.array_equal(native.mems[:, :native.mem_total], lowered.mems[:, :native.mem_total])


def test_corrupted_netlists():
    rtbuild.build()
    bases = _bases()
    rng = np.random.default_rng(2024)
    accepted = simulated = 0
    for it in range(1500):
        b = _corrupt(bytearray(bases[it % len(bases)]), rng)
        try:
            rt.rteaal_design_lower(b)
            lib_ok = True
        except rt.RteaalError as e:
            assert e.code == rt.RTEAAL_E_FORMAT, (it, str(e))
            lib_ok = False
        try:
            oracle.OracleSim(b, 1)
            orc_ok = True
        except ValueError:                          # the oracle's format error
            orc_ok = False
        assert lib_ok == orc_ok, it
        accepted += lib_ok
        if not lib_ok:                              # every host-only call refuses it alike
            for call in (lambda: rt.rteaal_design_single_clock(b, 1), lambda: rt.rteaal_design_rows(b, 1),
                         lambda: rt.rteaal_design_specialized_source(b)):
                try:
                    call()
                    raise AssertionError("accepted by one host-only call only: %d" % it)
                except rt.RteaalError as e:
                    assert e.code == rt.RTEAAL_E_FORMAT, (it, str(e))
        if lib_ok:
            nl = synth.Netlist.from_bytes(b)
            low, _ = rt.rteaal_design_lowered_netlist(b, nl.n_signals)
            rt.rteaal_design_rows(b, synth.Netlist.from_bytes(low).n_signals)
            assert "rteaal_spec" in rt.rteaal_design_specialized_source(b)
            rt.rteaal_design_single_clock(b, nl.n_signals)
            for fuse in (False, True):
                _lowering_simulates_alike(b, nl, fuse, it)
            if not nl.n_domains:                    # the restatements have no clock domains
                check(nl)
                _same_as_pyeval(b, nl, rng)
                simulated += 1
    assert 0 < accepted < 1500          # both outcomes occur
    assert simulated >= 50

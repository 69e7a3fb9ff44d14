"""The netlist-to-tensor lowering checked on the host (no GPU), through
rteaal_design_lower: the layer count and every layer's op count against the
levelisation restated from the netlist (Sec. 4.2), the compact state size
against the width classes, the copies the clock edge needs, operator fusion
against its absorption rule (App. B.1), and the (layer, opcode, width) grouping
against the keys that occur."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import OP, Builder, DesignSpec
from tests.netlist_rules import class_bytes, edge_copies, effective_args, fused_away, is_wide, levels


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()


def expected(nl: synth.Netlist, fuse: bool) -> dict:
    gone = fused_away(nl) if fuse else set()
    lv = levels(nl, gone)
    copies = edge_copies(nl)
    widths = nl.signal_widths()
    n_layers = max([int(lv.max()) if nl.n_ops else 0] + ([1] if copies else []))
    layer_ops = np.zeros(n_layers, np.int64)
    for k in range(nl.n_ops):
        if lv[k] > 0:
            layer_ops[lv[k] - 1] += 1
    if copies:
        layer_ops[0] += len(copies)
    n_lowered = nl.n_ops - len(gone) + len(copies)
    state = sum(class_bytes(int(w)) for w in widths[:nl.op_base])
    state += sum(class_bytes(int(nl.op_width[k])) for k in range(nl.n_ops) if lv[k] > 0)
    state += sum(class_bytes(int(widths[x])) for x in copies)
    # grouping keys: (layer, operand list wider than three, wide (ops with at
    # most three operands only), opcode, width)
    keys = set()
    for k in range(nl.n_ops):
        if lv[k] > 0:
            a = effective_args(nl, k, gone)
            code = OP["MUXCHAIN"] if (nl.op_code[k] == OP["MUX"] and len(a) > 3) else int(nl.op_code[k])
            keys.add((int(lv[k]), len(a) > 3, len(a) <= 3 and is_wide(nl, k, a, widths), code, int(nl.op_width[k])))
    for x in copies:
        keys.add((1, False, int(widths[x]) > 32, OP["COPY"], int(widths[x])))
    return dict(n_layers=n_layers, layer_ops=layer_ops, n_lowered_ops=n_lowered,
                n_slots=nl.op_base + n_lowered, state_bytes_per_lane=state, n_fused=len(gone),
                keys=keys, n_copies=len(copies))


def check(nl: synth.Netlist, fuse: bool = False) -> dict:
    info, layer_ops = rt.rteaal_design_lower(nl.to_bytes(), fuse_mux_chains=fuse)
    e = expected(nl, fuse)
    assert info["n_signals"] == nl.n_signals and info["n_ops"] == nl.n_ops
    assert info["n_inputs"] == nl.n_inputs and info["n_regs"] == nl.n_regs
    assert info["n_mems"] == nl.n_mems and info["n_wports"] == nl.n_wports
    assert info["n_layers"] == e["n_layers"]
    assert np.array_equal(layer_ops.astype(np.int64), e["layer_ops"])
    assert info["max_layer_ops"] == (int(e["layer_ops"].max()) if e["n_layers"] else 0)
    assert info["n_lowered_ops"] == e["n_lowered_ops"] == int(layer_ops.sum())
    assert info["n_slots"] == e["n_slots"]
    assert info["state_bytes_per_lane"] == e["state_bytes_per_lane"]
    assert info["n_fused"] == e["n_fused"]
    assert info["op_operands"] == nl.args.size
    assert info["mem_words_total"] == int(nl.mem_words.sum())
    assert info["metadata_bytes"] == 0
    # a group is a run of one (layer, opcode, width) in the sorted op list; the
    # ops with more than three operands of a layer follow the others
    distinct_lcw = {(l, c, w) for (l, _x, _wd, c, w) in e["keys"]}
    assert len(distinct_lcw) <= info["n_groups"] <= len(e["keys"])
    return info


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_designs(seed):
    nl = synth.generate(DesignSpec(n_ops=3000 + 500 * seed, n_regs=120, depth=12 + 4 * seed, seed=seed,
                                   n_inputs=4, n_mems=seed, mem_words=8,
                                   input_widths=(8, 32, 1, 64)))
    info = check(nl)
    assert info["n_layers"] >= 12 + 4 * seed - 1


def test_counter_lfsr_and_memories():
    check(synth.generate(synth.spec_tiny(0)))
    check(synth.generate(DesignSpec(n_ops=800, n_regs=40, depth=8, seed=5, n_mems=3, mem_words=16,
                                    mem_read_ports=2, mem_write_ports=2)))


@pytest.mark.parametrize("fuse", [False, True])
def test_mux_chains(fuse):
    nl = synth.generate(DesignSpec(n_ops=4000, n_regs=150, depth=16, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7, n_mems=2,
                                   mem_words=8))
    info = check(nl, fuse)
    if fuse:
        assert info["n_fused"] > 150
        plain, _ = rt.rteaal_design_lower(nl.to_bytes())
        assert info["n_layers"] <= plain["n_layers"]      # a chain is one op: fewer or equal layers
    else:
        assert info["n_fused"] == 0


def test_edge_copies_and_degenerate_designs():
    b = Builder()
    i0 = b.input(8)
    i1 = b.input(64)
    k = b.const(16, 0xBEEF)
    r0, r1, r2, r3 = b.reg(8, init=3), b.reg(64), b.reg(16), b.reg(8)
    b.connect(r0, i0)
    b.connect(r1, i1)
    b.connect(r2, k)
    b.connect(r3, r0)
    info = check(b.build())
    assert info["n_layers"] == 1 and info["n_lowered_ops"] == 4     # one copy per edge source
    b = Builder()
    b.input(1)
    info = check(b.build())
    assert info["n_layers"] == 0 and info["n_lowered_ops"] == 0
    # the same source feeding two registers and a write port gets one copy
    b = Builder()
    i0 = b.input(8)
    en = b.input(1)
    m = b.mem(4, 8)
    ra, rb = b.reg(8), b.reg(8)
    b.connect(ra, i0)
    b.connect(rb, i0)
    b.write_port(m, en, i0, i0)
    info = check(b.build())
    assert info["n_lowered_ops"] == 2


def test_clock_domains_add_work_only_with_domains():
    b = Builder()
    i0 = b.input(8)
    r = b.reg(8)
    b.connect(r, b.op("ADD", 8, r, i0))
    single, _ = rt.rteaal_design_lower(b.build().to_bytes())
    b = Builder()
    i0 = b.input(8)
    r = b.reg(8)
    b.connect(r, b.op("ADD", 8, r, i0))
    b.clock(r, b.domain(4, 1))
    multi, _ = rt.rteaal_design_lower(b.build().to_bytes())
    assert single["n_lowered_ops"] == 1
    # the domain's enable (from a hidden cycle counter) and the register's hold
    # mux are lowered into ordinary ops; the caller's figures are unchanged
    assert multi["n_lowered_ops"] > single["n_lowered_ops"]
    assert multi["n_ops"] == single["n_ops"] == 1 and multi["n_regs"] == single["n_regs"] == 1


def test_malformed_netlist_is_a_format_error():
    good = synth.generate(DesignSpec(n_ops=50, n_regs=4, depth=4, seed=1)).to_bytes()
    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_design_lower(good[:-1])
    assert ei.value.code == rt.RTEAAL_E_FORMAT

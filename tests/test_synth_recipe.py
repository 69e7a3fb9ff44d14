"""The synthetic input recipe (the stand-ins for the paper's designs and
benchmark programs): generated designs have the sizes, depth, operation-class
mix, width mix, mean arity and operand-distance law the recipe states, the
when/else chains of the mux-heavy workload are what they claim to be, and the
stimulus seeds and cycle budgets have their stated ranges."""
import numpy as np
import pytest

import synth
from synth import OP, DesignSpec
from synth.gen import MIX_DEFAULT, MIX_SOC, WIDTHS_DEFAULT
from tests.netlist_rules import levels

CLASSES = {
    "logic": ["AND", "OR", "XOR", "NOT", "ANDR", "ORR", "XORR"],
    "addsub": ["ADD", "SUB"],
    "mul": ["MUL"],
    "shift": ["SHL", "SHR", "DSHL", "DSHR", "BITS", "CAT"],
    "compare": ["EQ", "NEQ", "LT", "LEQ", "GT", "GEQ"],
    "mux": ["MUX"],
}
ONE_BIT = ["EQ", "NEQ", "LT", "LEQ", "GT", "GEQ", "ANDR", "ORR", "XORR"]


def nominal_layers(spec: DesignSpec) -> np.ndarray:
    """Ops are spread evenly over layers 1..depth, in netlist order."""
    counts = np.full(spec.depth, spec.n_ops // spec.depth)
    counts[: spec.n_ops % spec.depth] += 1
    return np.repeat(np.arange(1, spec.depth + 1), counts)


def class_shares(nl: synth.Netlist) -> dict:
    return {c: float(np.isin(nl.op_code, [OP[o] for o in ops]).mean()) for c, ops in CLASSES.items()}


@pytest.fixture(scope="module")
def default_design():
    spec = DesignSpec(n_ops=40_000, n_regs=2_000, depth=40, seed=3)
    return spec, synth.generate(spec)


def test_sizes_and_depth(default_design):
    spec, nl = default_design
    # constants: the 16 drawn ones plus a 1-bit and an 8-bit fallback operand
    assert (nl.n_ops, nl.n_regs, nl.n_inputs, nl.n_consts) == (40_000, 2_000, 8, 16 + 2)
    assert int(levels(nl).max()) == spec.depth            # every nominal layer is realised
    assert (nl.reg_d >= nl.op_base).all()                 # register D: an op output


def test_operation_class_mix(default_design):
    _spec, nl = default_design
    got = class_shares(nl)
    for c, pct in MIX_DEFAULT.items():
        assert abs(got[c] - pct / 100) < 0.015, (c, got[c])


def test_width_mix(default_design):
    """Output widths follow the width mix, except compares and reductions (1 bit),
    CAT (sum of its operands) and BITS (hi - lo + 1)."""
    _spec, nl = default_design
    free = ~np.isin(nl.op_code, [OP[o] for o in ONE_BIT + ["CAT", "BITS"]])
    assert (nl.op_width[np.isin(nl.op_code, [OP[o] for o in ONE_BIT])] == 1).all()
    w = nl.op_width[free]
    for width, p in WIDTHS_DEFAULT.items():
        assert abs(float((w == width).mean()) - p) < 0.015, width
    rw = nl.reg_width
    for width, p in WIDTHS_DEFAULT.items():
        assert abs(float((rw == width).mean()) - p) < 0.04, width


def test_mean_arity(default_design):
    # mix x arity: logic 0.30 x (0.84 x 2 + 0.16 x 1) + add/sub 0.15 x 2 + mul 0.05 x 2
    # + shift 0.15 x (6/9 x 1 + 3/9 x 2) + compare 0.10 x 2 + mux 0.25 x 3 = 2.102
    _spec, nl = default_design
    assert abs(float(np.diff(nl.op_argoff).mean()) - 2.102) < 0.02


def test_operand_distance_law(default_design):
    """An operand of an op on nominal layer L comes from layer L - d with
    P(d) = 2^-d (layers at or below 0 are the pool)."""
    spec, nl = default_design
    lay = nominal_layers(spec)
    src_layer = np.zeros(nl.n_signals, np.int64)
    src_layer[nl.op_base:] = lay
    d = []
    for k in np.flatnonzero(lay > 8):
        if nl.op_code[k] in (OP["MUL"], OP["CAT"]):
            continue                                        # operands re-drawn for width limits
        for x in nl.op_args(int(k)):
            d.append(lay[k] - src_layer[x] if x >= nl.op_base else 99)
    d = np.array(d)
    for j in range(1, 5):
        assert abs(float((d == j).mean()) - 2.0 ** -j) < 0.01, j


def test_soc_mix():
    nl = synth.generate(DesignSpec(n_ops=30_000, n_regs=1_000, depth=30, seed=8, mix=dict(MIX_SOC)))
    got = class_shares(nl)
    assert abs(got["mux"] - 0.40) < 0.015 and abs(got["compare"] - 0.15) < 0.015
    rest = 1 - 0.40 - 0.15
    for c in ["logic", "addsub", "mul", "shift"]:
        assert abs(got[c] - rest * MIX_DEFAULT[c] / 65) < 0.015, c


def chain_fraction(frac: float) -> float:
    """Share of the MUXes (above layer 1) whose false operand is a MUX of the
    previous layer, read by nothing else (not even a register or a write port)
    and at least as wide: the shape operator fusion absorbs."""
    spec = DesignSpec(n_ops=30_000, n_regs=1_000, depth=30, n_inputs=4, seed=9, mix=dict(MIX_SOC),
                      mux_chain_frac=frac, n_mems=2, mem_words=8, input_widths=(8, 32, 1, 64))
    nl = synth.generate(spec)
    fan = np.zeros(nl.n_signals, np.int64)
    np.add.at(fan, nl.args.astype(np.int64), 1)
    np.add.at(fan, nl.reg_d.astype(np.int64), 1)
    np.add.at(fan, nl.wport[:, 1:].reshape(-1).astype(np.int64), 1)
    lay = nominal_layers(spec)
    muxes = np.flatnonzero((nl.op_code == OP["MUX"]) & (lay > 1))
    chained = 0
    for k in muxes:
        f = int(nl.op_args(int(k))[2])
        j = f - nl.op_base
        chained += bool(f >= nl.op_base and nl.op_code[j] == OP["MUX"] and lay[j] == lay[k] - 1
                        and fan[f] == 1 and nl.op_width[j] >= nl.op_width[k])
    return chained / muxes.size


def test_when_else_chains():
    """mux_chain_frac: a chosen MUX takes as false operand a MUX of the previous
    layer that no other op reads, as far as the previous layer has such MUXes
    left; without it, chains are rare accidents of the random DAG."""
    assert chain_fraction(0.0) < 0.05
    assert chain_fraction(0.6) > 0.2


def test_stimulus_seeds_and_budgets():
    xs = synth.xorshift_seeds(2, 32, 4096)
    assert xs.shape == (32, 4096) and (xs != 0).all()        # 0 is xorshift64's fixed point
    assert np.unique(xs).size == xs.size
    b = synth.cycle_budgets(2, 4096, 1000, 100_000)
    assert b.min() >= 1000 and b.max() <= 100_000
    assert abs(float(b.mean()) - 50_500) < 1_500             # uniform on [1k, 100k]

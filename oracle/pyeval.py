"""Pure-Python reference evaluator -- TEST INFRASTRUCTURE ONLY.

A second, independently written statement of the operation semantics (the
readings listed in include/rteaal.h) using Python's unbounded integers and
``% 2**w`` instead of 64-bit wraparound, masks and shift guards.  A mistake in
oracle.c's overflow, masking or shift handling shows up as a disagreement
with this file.  Also a complete (slow) cycle simulator for tiny circuits,
used for brute force over every input assignment.
"""
from __future__ import annotations

from synth.netlist import OP, Netlist


def _m(x: int, w: int) -> int:
    return x % (1 << w)


def op_value(code: int, width: int, p0: int, p1: int, xs: list[int], mem=None) -> int:
    """Value of one operation from its operand values (O order)."""
    if code == OP["COPY"]:
        r = xs[0]
    elif code == OP["AND"]:
        r = xs[0]
        for x in xs[1:]:
            r = r & x
    elif code == OP["OR"]:
        r = xs[0]
        for x in xs[1:]:
            r = r | x
    elif code == OP["XOR"]:
        r = xs[0]
        for x in xs[1:]:
            r = r ^ x
    elif code == OP["NOT"]:
        r = (1 << 64) - 1 - xs[0]                     # 64-bit complement of a zero-extended value
    elif code == OP["ADD"]:
        r = sum(xs)
    elif code == OP["SUB"]:
        r = xs[0] - xs[1]
    elif code == OP["MUL"]:
        r = 1
        for x in xs:
            r = r * x
    elif code == OP["SHL"]:
        r = xs[0] * 2 ** p0
    elif code == OP["SHR"]:
        r = xs[0] // 2 ** p0
    elif code == OP["DSHL"]:
        r = xs[0] * 2 ** xs[1] if xs[1] < 128 else 0  # any amount >= 64 leaves no bit below 2^64
    elif code == OP["DSHR"]:
        r = xs[0] // 2 ** xs[1] if xs[1] < 128 else 0
    elif code == OP["BITS"]:
        hi, lo = p0, p1
        r = (xs[0] // 2 ** lo) % 2 ** (hi - lo + 1)
    elif code == OP["CAT"]:
        r = (xs[0] * 2 ** p0) | xs[1]
    elif code == OP["EQ"]:
        r = int(xs[0] == xs[1])
    elif code == OP["NEQ"]:
        r = int(xs[0] != xs[1])
    elif code == OP["LT"]:
        r = int(xs[0] < xs[1])
    elif code == OP["LEQ"]:
        r = int(xs[0] <= xs[1])
    elif code == OP["GT"]:
        r = int(xs[0] > xs[1])
    elif code == OP["GEQ"]:
        r = int(xs[0] >= xs[1])
    elif code == OP["MUX"]:
        r = xs[1] if xs[0] % 2 == 1 else xs[2]
    elif code == OP["ANDR"]:
        r = int(xs[0] % 2 ** p0 == 2 ** p0 - 1)
    elif code == OP["ORR"]:
        r = int(xs[0] != 0)
    elif code == OP["XORR"]:
        r = bin(xs[0]).count("1") % 2
    elif code == OP["MEMRD"]:
        words = mem[p0 + 256 * p1]
        r = words[xs[0] % len(words)]
    elif code == OP["MUXCHAIN"]:
        r = xs[-1]
        for i in range((len(xs) - 1) // 2):
            if xs[2 * i] % 2 == 1:
                r = xs[2 * i + 1]
                break
    else:
        raise ValueError("unknown opcode %d" % code)
    return _m(r, width)


class PySim:
    """One instance of a netlist, simulated with Python ints."""

    def __init__(self, nl: Netlist):
        self.nl = nl
        self.v = [0] * nl.n_signals
        for c in range(nl.n_consts):
            self.v[nl.const_base + c] = _m(int(nl.const_value[c]), int(nl.const_width[c]))
        self.mem = [[0] * int(nl.mem_words[m]) for m in range(nl.n_mems)]
        self.args = [[int(a) for a in nl.op_args(k)] for k in range(nl.n_ops)]

    def cycle(self, inputs: list[int], reset: bool = False):
        nl, v = self.nl, self.v
        for j, x in enumerate(inputs):
            v[j] = _m(int(x), int(nl.input_width[j]))
        for k in range(nl.n_ops):
            v[nl.op_base + k] = op_value(int(nl.op_code[k]), int(nl.op_width[k]), int(nl.op_p0[k]),
                                         int(nl.op_p1[k]), [v[a] for a in self.args[k]], self.mem)
        nxt = [_m(int(nl.reg_init[r]) if reset else v[int(nl.reg_d[r])], int(nl.reg_width[r]))
               for r in range(nl.n_regs)]
        for p in range(nl.n_wports):
            m, en, addr, data = (int(x) for x in nl.wport[p])
            if v[en] % 2 == 1:
                self.mem[m][v[addr] % len(self.mem[m])] = _m(v[data], int(nl.mem_width[m]))
        for r in range(nl.n_regs):
            v[nl.reg_base + r] = nxt[r]

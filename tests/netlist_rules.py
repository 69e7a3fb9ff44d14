"""The lowering's structural rules restated over a netlist in plain Python, for
host-side checks of the lowering and of operator fusion.  No simulation
arithmetic lives here."""
from __future__ import annotations

import numpy as np

import synth
from synth import OP


def fused_away(nl: synth.Netlist) -> set:
    """The muxes the fusion rule absorbs (App. B.1): walking the ops from the top
    of the topological order down, a MUX whose false operand (O = 2) is a MUX
    read nowhere else and at least as wide as the chain's head joins the chain.
    Returns signal ids."""
    fan = np.zeros(nl.n_signals, np.int64)
    np.add.at(fan, nl.args.astype(np.int64), 1)
    np.add.at(fan, nl.reg_d.astype(np.int64), 1)
    if nl.n_wports:
        np.add.at(fan, nl.wport[:, 1:].reshape(-1).astype(np.int64), 1)
    gone = set()
    for k in range(nl.n_ops - 1, -1, -1):
        if k in gone or nl.op_code[k] != OP["MUX"]:
            continue
        w0 = int(nl.op_width[k])
        cur = k
        while True:
            x = int(nl.op_args(cur)[2])
            j = x - nl.op_base
            if x < nl.op_base or nl.op_code[j] != OP["MUX"] or fan[x] != 1 or nl.op_width[j] < w0:
                break
            gone.add(j)
            cur = j
    return {nl.op_base + j for j in gone}


def effective_args(nl: synth.Netlist, k: int, gone: set) -> list[int]:
    """Operands of op k after fusion: a chain head reads every selector and true
    value of its chain, then the last false operand."""
    a = [int(x) for x in nl.op_args(k)]
    if nl.op_code[k] != OP["MUX"] or a[2] not in gone:
        return a
    out = []
    while True:
        out += a[:2]
        if a[2] not in gone:
            return out + [a[2]]
        a = [int(x) for x in nl.op_args(a[2] - nl.op_base)]


def levels(nl: synth.Netlist, gone: set = frozenset()) -> np.ndarray:
    """Layer of every op (Sec. 4.2): inputs, registers and constants are layer 0,
    an op is one layer above its deepest operand; absorbed muxes get -1."""
    lv = np.zeros(nl.n_signals, np.int64)
    out = np.full(nl.n_ops, -1, np.int64)
    for k in range(nl.n_ops):
        if nl.op_base + k in gone:
            continue
        lv[nl.op_base + k] = 1 + max(lv[x] for x in effective_args(nl, k, gone))
        out[k] = lv[nl.op_base + k]
    return out


def edge_copies(nl: synth.Netlist) -> list[int]:
    """Signals the clock edge reads that are not op outputs (register D and
    write-port enable / address / data fed by an input, register or constant):
    each gets one copy op in layer 1."""
    read = [int(x) for x in nl.reg_d]
    if nl.n_wports:
        read += [int(x) for x in nl.wport[:, 1:].reshape(-1)]
    return sorted({x for x in read if x < nl.op_base})


def class_bytes(width: int) -> int:
    """Bytes per lane of a row holding a signal of this width (1, 2, 4 or 8)."""
    return 1 if width <= 8 else 2 if width <= 16 else 4 if width <= 32 else 8


def is_wide(nl: synth.Netlist, k: int, args: list[int], w: np.ndarray) -> bool:
    """Op k is evaluated in 64-bit arithmetic (not narrow): its result or an
    operand is wider than 32 bits, it reads a memory, or it is a BITS reaching
    bit 32 or an ANDR over more than 32 bits.  w: the netlist's signal widths."""
    code = int(nl.op_code[k])
    return (int(nl.op_width[k]) > 32 or code == OP["MEMRD"] or (code == OP["BITS"] and nl.op_p0[k] >= 32)
            or (code == OP["ANDR"] and nl.op_p0[k] > 32) or any(int(w[x]) > 32 for x in args))

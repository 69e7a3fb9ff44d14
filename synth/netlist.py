"""In-memory netlist and its binary serialisation ("RTLN" version 1).

A netlist is the dataflow graph of a synchronous single-clock design (Sec. 2.1,
Fig. 1 of the paper): primary inputs, registers, constants, combinational
operations in topological order, and optional register-file memories.  This
module only stores and (de)serialises it; it holds no evaluation arithmetic.
The byte layout is specified in ``include/rteaal.h`` (section "Netlist
format"), which is what ``rteaal_design_load`` parses.

Signal numbering is implicit:
    [0, n_inputs)                         primary inputs
    [n_inputs, +n_regs)                   register outputs (Q)
    [.., +n_consts)                       constants
    [.., +n_ops)                          operation outputs, in topological order
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

import numpy as np

MAGIC = 0x4E4C5452  # b"RTLN" little-endian
VERSION = 1
HEADER = struct.Struct("<10I")

# Opcodes (u8).  Semantics are defined in include/rteaal.h.
OP = dict(
    COPY=0, AND=1, OR=2, XOR=3, NOT=4, ADD=5, SUB=6, MUL=7,
    SHL=8, SHR=9, DSHL=10, DSHR=11, BITS=12, CAT=13,
    EQ=14, NEQ=15, LT=16, LEQ=17, GT=18, GEQ=19,
    MUX=20, ANDR=21, ORR=22, XORR=23, MEMRD=24, MUXCHAIN=25,
)
OPNAME = {v: k for k, v in OP.items()}
N_OPCODES = 26

# Fixed arity per opcode; -2 = variadic >= 2 (fold in O order); -3 = odd >= 3.
ARITY = {
    OP["COPY"]: 1, OP["AND"]: -2, OP["OR"]: -2, OP["XOR"]: -2, OP["NOT"]: 1,
    OP["ADD"]: -2, OP["SUB"]: 2, OP["MUL"]: -2, OP["SHL"]: 1, OP["SHR"]: 1,
    OP["DSHL"]: 2, OP["DSHR"]: 2, OP["BITS"]: 1, OP["CAT"]: 2,
    OP["EQ"]: 2, OP["NEQ"]: 2, OP["LT"]: 2, OP["LEQ"]: 2, OP["GT"]: 2, OP["GEQ"]: 2,
    OP["MUX"]: 3, OP["ANDR"]: 1, OP["ORR"]: 1, OP["XORR"]: 1, OP["MEMRD"]: 1,
    OP["MUXCHAIN"]: -3,
}


@dataclass
class Netlist:
    input_width: np.ndarray                      # u8 [n_inputs]
    reg_width: np.ndarray                        # u8 [n_regs]
    reg_d: np.ndarray                            # u32 [n_regs]  signal id of D
    reg_init: np.ndarray                         # u64 [n_regs]
    const_width: np.ndarray                      # u8 [n_consts]
    const_value: np.ndarray                      # u64 [n_consts]
    op_code: np.ndarray                          # u8 [n_ops]
    op_width: np.ndarray                         # u8 [n_ops]
    op_p0: np.ndarray                            # u8 [n_ops]
    op_p1: np.ndarray                            # u8 [n_ops]
    op_argoff: np.ndarray                        # u32 [n_ops+1] (CSR into args)
    args: np.ndarray                             # u32 [n_args]  operand signal ids, O order
    mem_words: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))  # u32 [n_mems]
    mem_width: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))   # u8 [n_mems]
    wport: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.uint32))  # u32 [n_wports][mem,en,addr,data]
    # optional clock domains: per domain a period (power of two) and a phase in
    # base-clock cycles; per register its domain (no domains: one base clock)
    dom_period: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))  # u32 [n_domains]
    dom_phase: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))   # u32 [n_domains]
    reg_domain: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))   # u8 [n_regs] if domains

    # ---- sizes -------------------------------------------------------------
    @property
    def n_inputs(self) -> int: return int(self.input_width.size)
    @property
    def n_regs(self) -> int: return int(self.reg_width.size)
    @property
    def n_consts(self) -> int: return int(self.const_width.size)
    @property
    def n_ops(self) -> int: return int(self.op_code.size)
    @property
    def n_mems(self) -> int: return int(self.mem_words.size)
    @property
    def n_wports(self) -> int: return int(self.wport.shape[0])
    @property
    def n_domains(self) -> int: return int(self.dom_period.size)
    @property
    def n_signals(self) -> int: return self.n_inputs + self.n_regs + self.n_consts + self.n_ops
    @property
    def reg_base(self) -> int: return self.n_inputs
    @property
    def const_base(self) -> int: return self.n_inputs + self.n_regs
    @property
    def op_base(self) -> int: return self.n_inputs + self.n_regs + self.n_consts

    def signal_widths(self) -> np.ndarray:
        return np.concatenate([self.input_width, self.reg_width, self.const_width,
                               self.op_width]).astype(np.uint8)

    def op_args(self, k: int) -> np.ndarray:
        return self.args[self.op_argoff[k]:self.op_argoff[k + 1]]

    # ---- serialisation -----------------------------------------------------
    def to_bytes(self) -> bytes:
        nd = self.n_domains
        hdr = HEADER.pack(MAGIC, VERSION, self.n_inputs, self.n_regs, self.n_consts,
                          self.n_ops, self.n_mems, self.n_wports, int(self.args.size), nd)
        parts = [hdr,
                 np.ascontiguousarray(self.reg_init, "<u8").tobytes(),
                 np.ascontiguousarray(self.const_value, "<u8").tobytes(),
                 np.ascontiguousarray(self.reg_d, "<u4").tobytes(),
                 np.ascontiguousarray(self.op_argoff, "<u4").tobytes(),
                 np.ascontiguousarray(self.args, "<u4").tobytes(),
                 np.ascontiguousarray(self.mem_words, "<u4").tobytes(),
                 np.ascontiguousarray(self.wport.reshape(-1, 4), "<u4").tobytes(),
                 np.ascontiguousarray(self.dom_period, "<u4").tobytes() if nd else b"",
                 np.ascontiguousarray(self.dom_phase, "<u4").tobytes() if nd else b"",
                 np.ascontiguousarray(self.input_width, "u1").tobytes(),
                 np.ascontiguousarray(self.reg_width, "u1").tobytes(),
                 np.ascontiguousarray(self.const_width, "u1").tobytes(),
                 np.ascontiguousarray(self.op_code, "u1").tobytes(),
                 np.ascontiguousarray(self.op_width, "u1").tobytes(),
                 np.ascontiguousarray(self.op_p0, "u1").tobytes(),
                 np.ascontiguousarray(self.op_p1, "u1").tobytes(),
                 np.ascontiguousarray(self.mem_width, "u1").tobytes(),
                 np.ascontiguousarray(self.reg_domain, "u1").tobytes() if nd else b""]
        return b"".join(parts)

    @staticmethod
    def from_bytes(buf: bytes) -> "Netlist":
        (magic, ver, ni, nr, nc, no, nm, nw, na, nd) = HEADER.unpack_from(buf, 0)
        if magic != MAGIC or ver != VERSION:
            raise ValueError("not an RTLN v1 netlist")
        off = HEADER.size

        def take(dtype, count):
            nonlocal off
            a = np.frombuffer(buf, dtype=dtype, count=count, offset=off).copy()
            off += a.nbytes
            return a

        reg_init = take("<u8", nr).astype(np.uint64)
        const_value = take("<u8", nc).astype(np.uint64)
        reg_d = take("<u4", nr).astype(np.uint32)
        op_argoff = take("<u4", no + 1).astype(np.uint32)
        args = take("<u4", na).astype(np.uint32)
        mem_words = take("<u4", nm).astype(np.uint32)
        wport = take("<u4", 4 * nw).astype(np.uint32).reshape(nw, 4)
        dom_period = take("<u4", nd).astype(np.uint32)
        dom_phase = take("<u4", nd).astype(np.uint32)
        input_width = take("u1", ni)
        reg_width = take("u1", nr)
        const_width = take("u1", nc)
        op_code = take("u1", no)
        op_width = take("u1", no)
        op_p0 = take("u1", no)
        op_p1 = take("u1", no)
        mem_width = take("u1", nm)
        reg_domain = take("u1", nr if nd else 0)
        if off != len(buf):
            raise ValueError("trailing bytes in netlist")
        return Netlist(input_width, reg_width, reg_d, reg_init, const_width, const_value,
                       op_code, op_width, op_p0, op_p1, op_argoff, args,
                       mem_words, mem_width, wport, dom_period, dom_phase, reg_domain)


class Builder:
    """Incremental netlist construction for small hand-written circuits (tests, examples)."""

    def __init__(self):
        self.inputs: list[int] = []
        self.regs: list[list] = []          # [width, d, init]
        self.consts: list[list] = []        # [width, value]
        self.ops: list[tuple] = []          # (code, width, p0, p1, args-as-handles)
        self.mems: list[tuple] = []         # (words, width)
        self.wports: list[tuple] = []       # (mem, en, addr, data) as handles
        self.domains: list[tuple] = []      # (period, phase)
        self.reg_dom: dict[int, int] = {}   # register index -> domain

    # Handles are ("i", k), ("r", k), ("c", k), ("o", k); resolved at build().
    def input(self, width: int):
        self.inputs.append(width)
        return ("i", len(self.inputs) - 1)

    def reg(self, width: int, init: int = 0):
        self.regs.append([width, None, init])
        return ("r", len(self.regs) - 1)

    def const(self, width: int, value: int):
        self.consts.append([width, value])
        return ("c", len(self.consts) - 1)

    def op(self, name: str, width: int, *args, p0: int = 0, p1: int = 0):
        self.ops.append((OP[name], width, p0, p1, tuple(args)))
        return ("o", len(self.ops) - 1)

    def mem(self, words: int, width: int = 64) -> int:
        self.mems.append((words, width))
        return len(self.mems) - 1

    def write_port(self, mem: int, en, addr, data):
        self.wports.append((mem, en, addr, data))

    def connect(self, reg, d):
        self.regs[reg[1]][1] = d

    def domain(self, period: int, phase: int = 0) -> int:
        """A clock domain ticking when (t + phase) mod period == 0 (t: cycles since reset)."""
        self.domains.append((period, phase))
        return len(self.domains) - 1

    def clock(self, reg, domain: int):
        self.reg_dom[reg[1]] = domain

    def build(self) -> Netlist:
        ni, nr, nc = len(self.inputs), len(self.regs), len(self.consts)
        base = {"i": 0, "r": ni, "c": ni + nr, "o": ni + nr + nc}

        def sid(h):
            return base[h[0]] + h[1]

        argoff = [0]
        args: list[int] = []
        for (_c, _w, _p0, _p1, a) in self.ops:
            args.extend(sid(x) for x in a)
            argoff.append(len(args))
        for r in self.regs:
            if r[1] is None:
                raise ValueError("register without D connection")
        return Netlist(
            input_width=np.array(self.inputs, np.uint8),
            reg_width=np.array([r[0] for r in self.regs], np.uint8),
            reg_d=np.array([sid(r[1]) for r in self.regs], np.uint32),
            reg_init=np.array([r[2] for r in self.regs], np.uint64),
            const_width=np.array([c[0] for c in self.consts], np.uint8),
            const_value=np.array([c[1] for c in self.consts], np.uint64),
            op_code=np.array([o[0] for o in self.ops], np.uint8),
            op_width=np.array([o[1] for o in self.ops], np.uint8),
            op_p0=np.array([o[2] for o in self.ops], np.uint8),
            op_p1=np.array([o[3] for o in self.ops], np.uint8),
            op_argoff=np.array(argoff, np.uint32),
            args=np.array(args, np.uint32),
            mem_words=np.array([m[0] for m in self.mems], np.uint32),
            mem_width=np.array([m[1] for m in self.mems], np.uint8),
            wport=np.array([[m, sid(e), sid(a), sid(d)] for (m, e, a, d) in self.wports],
                           np.uint32).reshape(-1, 4),
            dom_period=np.array([d[0] for d in self.domains], np.uint32),
            dom_phase=np.array([d[1] for d in self.domains], np.uint32),
            reg_domain=(np.array([self.reg_dom.get(r, 0) for r in range(nr)], np.uint8)
                        if self.domains else np.zeros(0, np.uint8)),
        )

    def sid(self, h) -> int:
        ni, nr, nc = len(self.inputs), len(self.regs), len(self.consts)
        return {"i": 0, "r": ni, "c": ni + nr, "o": ni + nr + nc}[h[0]] + h[1]

"""The paper's Einsum cascade, evaluated literally -- TEST INFRASTRUCTURE ONLY.

Follows Sec. 4 of the paper step by step, for small circuits:

  * levelisation (Sec. 4.2): layer of an op = 1 + max(layer of its operands),
    primary inputs / registers / constants form layer 0;
  * identity operations (Sec. 4.2, Fig. "df_preprocess"): every value consumed
    more than one layer later, or at the clock edge, is forwarded layer by
    layer so that layer i+1 reads only the outputs of layer i;
  * per layer i, the operation input mask OIM_i with ranks [S, N, O, R]
    (one-hot N and R, dense O in ascending order, Sec. 4.1 and 4.3);
  * per cycle, Cascade 1 in the loop order [I, S, N, O, R] of Alg. 3:
        OI       = LI_i . OIM_i           (map, take-left)
        LO_i     = op_u[n] then op_r[n]   (map compute, reduce compute in O order;
                                           the first map temporary is copied)
        LO_sel_i = op_s[n] on the O-fiber (populate coordinate operator)
        LI_{i+1} = LO_i / LO_sel_i        (ANY reduce; the two never overlap)
  * the clock edge commits registers from LI_I.

Readings (also stated in include/rteaal.h): the operation type n is the tuple
(opcode, width, p0, p1); a result is masked to the type's width after op_r /
op_s; memory reads are a unary op_u that also reads the memory state (the paper
has no memories).  This evaluator is independent of oracle.c; it borrows only
the per-operation definitions of :mod:`oracle.pyeval`, so a disagreement with
oracle.c points at the cascade structure (levels, identities, O order, edge).
"""
from __future__ import annotations

from synth.netlist import OP, Netlist

from .pyeval import op_value

IDENTITY = ("identity",)
UNARY = {OP["COPY"], OP["NOT"], OP["SHL"], OP["SHR"], OP["BITS"], OP["ANDR"], OP["ORR"],
         OP["XORR"], OP["MEMRD"]}
SELECT = {OP["MUX"], OP["MUXCHAIN"]}                  # n_sel
REDUCIBLE = {OP["AND"], OP["OR"], OP["XOR"], OP["ADD"], OP["SUB"], OP["MUL"], OP["DSHL"],
             OP["DSHR"], OP["CAT"], OP["EQ"], OP["NEQ"], OP["LT"], OP["LEQ"], OP["GT"], OP["GEQ"]}


def levelize(nl: Netlist) -> list[int]:
    """Layer (longest path from layer 0) of every signal."""
    lvl = [0] * nl.n_signals
    for k in range(nl.n_ops):
        a = nl.op_args(k)
        lvl[nl.op_base + k] = 1 + max((lvl[int(x)] for x in a), default=0)
    return lvl


class CascadeSim:
    def __init__(self, nl: Netlist):
        self.nl = nl
        lvl = levelize(nl)
        self.lvl = lvl
        I = max(lvl[nl.op_base:], default=0)
        self.I = I
        # last LI index in which each signal must be present
        need = [-1] * nl.n_signals
        for k in range(nl.n_ops):
            for x in nl.op_args(k):
                need[int(x)] = max(need[int(x)], lvl[nl.op_base + k] - 1)
        edge = [int(d) for d in nl.reg_d] + [int(s) for p in nl.wport for s in p[1:]]
        for x in edge:
            need[x] = I
        # LI_0: rank R = the pool (inputs, registers, constants), coordinate = signal id
        self.li0 = list(range(nl.op_base))
        # per layer i: list of (n, sig_or_None, [(o, r)]) in S order, and the LO coordinates
        self.layers = []
        li = self.li0
        for i in range(I):
            rpos = {sig: r for r, sig in enumerate(li)}
            S = []
            lo_sigs = []
            for k in range(nl.n_ops):                    # effectual ops of level i+1
                sig = nl.op_base + k
                if lvl[sig] != i + 1:
                    continue
                n = (int(nl.op_code[k]), int(nl.op_width[k]), int(nl.op_p0[k]), int(nl.op_p1[k]))
                S.append((n, sig, [(o, rpos[int(x)]) for o, x in enumerate(nl.op_args(k))]))
                lo_sigs.append(sig)
            for sig in li:                               # identity ops (forwarding)
                if need[sig] >= i + 1:
                    S.append((IDENTITY, sig, [(0, rpos[sig])]))
                    lo_sigs.append(sig)
            self.layers.append(S)
            li = lo_sigs
        self.li_final = li
        self.n_identity = sum(1 for S in self.layers for e in S if e[0] is IDENTITY)
        # state (one instance)
        self.v = [0] * nl.n_signals
        for c in range(nl.n_consts):
            self.v[nl.const_base + c] = int(nl.const_value[c]) % (1 << int(nl.const_width[c]))
        self.mem = [[0] * int(nl.mem_words[m]) for m in range(nl.n_mems)]

    # custom operators of Cascade 1 ------------------------------------------------
    def op_u(self, n, x):
        if n is IDENTITY or n[0] not in UNARY:
            return x                                     # pass-through
        return op_value(n[0], 64, n[2], n[3], [x], self.mem)

    def op_r(self, n, prev, x):
        if n is IDENTITY or n[0] not in REDUCIBLE:
            return x                                     # copy the map temporary
        return op_value(n[0], 64, n[2], n[3], [prev, x])

    def op_s(self, n, sel_inputs):
        return op_value(n[0], 64, n[2], n[3], sel_inputs)

    def cycle(self, inputs: list[int], reset: bool = False):
        nl, v = self.nl, self.v
        for j, x in enumerate(inputs):
            v[j] = int(x) % (1 << int(nl.input_width[j]))
        LI = [v[sig] for sig in self.li0]
        for S in self.layers:                            # rank I (iterative)
            LO = [None] * len(S)
            for s, (n, sig, fiber) in enumerate(S):      # rank S, then N (one-hot)
                sel_inputs = []
                for o, r in fiber:                       # rank O ascending, R one-hot
                    oi = LI[r]                           # OI = LI . OIM  (take-left)
                    sel_inputs.append(oi)
                    map_tmp = self.op_u(n, oi)
                    LO[s] = map_tmp if LO[s] is None else self.op_r(n, LO[s], map_tmp)
                if n is not IDENTITY and n[0] in SELECT:
                    LO[s] = self.op_s(n, sel_inputs)     # LO_sel
                if n is not IDENTITY:
                    LO[s] %= 1 << n[1]
                    v[sig] = LO[s]
            LI = LO                                      # LI_{i+1} = LO_i (ANY)
        final = {sig: LI[r] for r, sig in enumerate(self.li_final)}
        if not self.layers:
            final = {sig: v[sig] for sig in self.li0}
        nxt = [(int(nl.reg_init[r]) if reset else final[int(nl.reg_d[r])]) % (1 << int(nl.reg_width[r]))
               for r in range(nl.n_regs)]
        for p in range(nl.n_wports):
            m, en, addr, data = (int(x) for x in nl.wport[p])
            if final[en] % 2 == 1:
                self.mem[m][final[addr] % len(self.mem[m])] = final[data] % (1 << int(nl.mem_width[m]))
        for r in range(nl.n_regs):
            v[nl.reg_base + r] = nxt[r]

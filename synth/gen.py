"""Seeded synthetic circuits and stimulus seeds.

Stands in for the paper's Chipyard designs (RocketChip, BOOM, Gemmini, SHA3;
Sec. 7.1; Table 1), which are not available: random layered dataflow graphs
whose scale matches or exceeds Table 1's effectual-operation counts.  This
module only *builds* netlists and draws random seeds; it evaluates nothing.

Every random draw comes from one counter-based stream: SplitMix64's output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``key + i * 0x9E3779B97F4A7C15``.  Being
counter based and written with numpy uint64 arithmetic, the same seed gives
the same netlist on any machine and numpy version.

Generator specification (fixed, versioned with GEN_VERSION):
  * layer 0 is the pool: primary inputs, register outputs and constants;
  * ``n_ops`` ops are spread evenly over layers 1..depth;
  * each operand of an op on nominal layer L comes from layer L-d with
    P(d) = 2^-d (d >= 1, geometric(0.5)); a layer index <= 0 means the pool;
    within the chosen layer the signal is uniform;
  * op classes follow the configured mix; within a class the opcode is drawn
    from fixed sub-weights (below);
  * output widths are drawn from the configured width distribution, except
    compares / reductions (1 bit), CAT (w_a + w_b), BITS (hi - lo + 1);
  * MUL operands are re-drawn until both are <= 32 bits wide; CAT operands
    until w_a + w_b <= 64 (after 32 re-draws a narrow pool constant is used);
  * each register's D is a uniformly chosen op output; register widths follow
    the width distribution; memories' write-port signals are uniform op outputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .netlist import OP, Netlist

GEN_VERSION = 1
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based stream: draw i is mix(key + (i+1) * gamma)."""

    def __init__(self, seed: int, stream: int = 0):
        with np.errstate(over="ignore"):
            k = splitmix64_mix(np.array([np.uint64(seed & (2**64 - 1))], np.uint64) * GAMMA
                               + np.uint64(stream & (2**64 - 1)))
        self.key = np.uint64(k[0])
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return splitmix64_mix(self.key + i * GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def below(self, bound, n: int) -> np.ndarray:
        """Uniform integers in [0, bound) (bound scalar or array, all >= 1)."""
        b = np.asarray(bound, dtype=np.float64)
        r = np.floor(self.uniform(n) * b).astype(np.int64)
        return np.minimum(r, np.asarray(bound, np.int64) - 1)

    def choice(self, values, probs, n: int) -> np.ndarray:
        p = np.asarray(probs, np.float64)
        c = np.cumsum(p / p.sum())
        idx = np.searchsorted(c, self.uniform(n), side="right")
        return np.asarray(values)[np.minimum(idx, len(values) - 1)]

    def geometric_half(self, n: int) -> np.ndarray:
        """d >= 1 with P(d) = 2^-d: one plus the trailing-zero count of a uniform word."""
        u = self.u64(n)
        with np.errstate(over="ignore"):
            low = u & (~u + np.uint64(1))
        d = np.where(u == 0, 64, np.log2(np.maximum(low, 1).astype(np.float64)).astype(np.int64))
        return 1 + d


# ---------------------------------------------------------------------------
# Configuration of a synthetic design
# ---------------------------------------------------------------------------
WIDTHS_DEFAULT = {1: 0.4, 8: 0.15, 16: 0.1, 32: 0.2, 64: 0.15}
# class mix in percent: logic, addsub, mul, shift (shift/bits/cat), compare, mux
MIX_DEFAULT = {"logic": 30, "addsub": 15, "mul": 5, "shift": 15, "compare": 10, "mux": 25}
# SoC-like mix: 40% mux, 15% compare, the rest scaled from the default mix
MIX_SOC = {"logic": 30 * 45 / 65, "addsub": 15 * 45 / 65, "mul": 5 * 45 / 65,
           "shift": 15 * 45 / 65, "compare": 15, "mux": 40}

_SUB = {
    "logic": ([OP["AND"], OP["OR"], OP["XOR"], OP["NOT"], OP["ANDR"], OP["ORR"], OP["XORR"]],
              [0.28, 0.28, 0.28, 0.06, 0.03, 0.03, 0.04]),
    "addsub": ([OP["ADD"], OP["SUB"]], [0.5, 0.5]),
    "mul": ([OP["MUL"]], [1.0]),
    "shift": ([OP["SHL"], OP["SHR"], OP["BITS"], OP["DSHL"], OP["DSHR"], OP["CAT"]],
              [2 / 9, 2 / 9, 2 / 9, 1 / 9, 1 / 9, 1 / 9]),
    "compare": ([OP["EQ"], OP["NEQ"], OP["LT"], OP["LEQ"], OP["GT"], OP["GEQ"]], [1 / 6] * 6),
    "mux": ([OP["MUX"]], [1.0]),
}
_ARITY = np.zeros(32, np.int64)
for _name, _a in [("AND", 2), ("OR", 2), ("XOR", 2), ("NOT", 1), ("ANDR", 1), ("ORR", 1),
                  ("XORR", 1), ("ADD", 2), ("SUB", 2), ("MUL", 2), ("SHL", 1), ("SHR", 1),
                  ("BITS", 1), ("DSHL", 2), ("DSHR", 2), ("CAT", 2), ("EQ", 2), ("NEQ", 2),
                  ("LT", 2), ("LEQ", 2), ("GT", 2), ("GEQ", 2), ("MUX", 3), ("MEMRD", 1)]:
    _ARITY[OP[_name]] = _a


@dataclass
class DesignSpec:
    n_ops: int
    n_regs: int
    depth: int
    n_inputs: int = 8
    n_consts: int = 16
    seed: int = 0
    widths: dict = field(default_factory=lambda: dict(WIDTHS_DEFAULT))
    mix: dict = field(default_factory=lambda: dict(MIX_DEFAULT))
    counter_lfsr: bool = False        # add the 32-bit counter and 16-bit Galois LFSR (taps 0xB400)
    n_mems: int = 0                   # register files (words x 64 bit)
    mem_words: int = 32
    mem_read_ports: int = 2
    mem_write_ports: int = 1
    input_widths: tuple | None = None  # explicit primary-input widths (overrides the draw)
    mux_chain_frac: float = 0.0       # P(a MUX takes a previous-layer MUX nothing else reads as its
                                      # false operand), capped by how many such MUXes are left


# Named workloads: the sizes the parity tests and the benchmark use.
def spec_tiny(seed: int = 0) -> DesignSpec:
    """2,000-op DAG over 64 registers, depth 20, plus counter and LFSR; 8 inputs."""
    return DesignSpec(n_ops=2000, n_regs=64, depth=20, n_inputs=8, seed=seed, counter_lfsr=True)


def spec_single(seed: int = 1) -> DesignSpec:
    """200k-op DAG, 20k registers, depth 60 (single-instance form)."""
    return DesignSpec(n_ops=200_000, n_regs=20_000, depth=60, n_inputs=8, seed=seed)


def spec_batch(seed: int = 2) -> DesignSpec:
    """1M-op DAG, 64k registers, depth 80, 32 inputs (batched form)."""
    return DesignSpec(n_ops=1_000_000, n_regs=65_536, depth=80, n_inputs=32, seed=seed)


def spec_soc(seed: int = 3) -> DesignSpec:
    """5M-op SoC-like DAG, depth 120, 256k registers, 64 register files of 32 x 64 bit."""
    return DesignSpec(n_ops=5_000_000, n_regs=262_144, depth=120, n_inputs=32, seed=seed,
                      mix=dict(MIX_SOC), n_mems=64, mem_words=32)


def spec_mux(seed: int = 4) -> DesignSpec:
    """1M-op control-heavy DAG (SoC mix, 40% mux) whose muxes chain with probability 0.6."""
    return DesignSpec(n_ops=1_000_000, n_regs=65_536, depth=80, n_inputs=32, seed=seed,
                      mix=dict(MIX_SOC), mux_chain_frac=0.6)


def spec_serving(n_ops: int, seed: int) -> DesignSpec:
    depth = {50_000: 40, 500_000: 80, 5_000_000: 120}.get(n_ops, 40)
    return DesignSpec(n_ops=n_ops, n_regs=max(1, n_ops // 20), depth=depth, n_inputs=8, seed=seed)


# ---------------------------------------------------------------------------
def generate(spec: DesignSpec) -> Netlist:
    rng = Rng(spec.seed, stream=0x5EED0000 + GEN_VERSION)
    wv = np.array(list(spec.widths.keys()), np.int64)
    wp = np.array(list(spec.widths.values()), np.float64)

    n_in, n_rand_regs, n_c = spec.n_inputs, spec.n_regs, spec.n_consts
    n_special_regs = 2 if spec.counter_lfsr else 0
    n_regs = n_rand_regs + n_special_regs

    input_width = rng.choice(wv, wp, n_in).astype(np.uint8)
    # the first input is forced narrow so that MUL / CAT fallbacks always exist
    if n_in:
        input_width[0] = 8
    if spec.input_widths is not None:
        input_width = np.array(spec.input_widths, np.uint8)
        assert input_width.size == n_in
    reg_width = rng.choice(wv, wp, n_regs).astype(np.uint8)
    reg_init = np.zeros(n_regs, np.uint64)

    const_width = rng.choice(wv, wp, n_c).astype(np.uint8)
    special_consts = []
    if spec.counter_lfsr:
        special_consts = [(32, 1), (16, 0xB400)]
    const_width = np.concatenate([const_width, np.array([1, 8], np.uint8),
                                  np.array([w for w, _ in special_consts], np.uint8)])
    cvals = rng.u64(const_width.size)
    cw = const_width.astype(np.uint64)
    cmask = np.where(cw >= 64, np.uint64(2**64 - 1),
                     (np.uint64(1) << np.minimum(cw, 63)) - np.uint64(1))
    const_value = cvals & cmask
    k0 = n_c  # index of the 1-bit fallback constant, k0+1 the 8-bit one
    for j, (w, v) in enumerate(special_consts):
        const_value[n_c + 2 + j] = v
    n_consts = const_width.size

    reg_base = n_in
    const_base = n_in + n_regs
    op_base = const_base + n_consts
    n_ops_total = spec.n_ops + (5 if spec.counter_lfsr else 0)
    n_signals = op_base + n_ops_total

    sig_width = np.zeros(n_signals, np.int64)
    sig_width[:n_in] = input_width
    sig_width[reg_base:reg_base + n_regs] = reg_width
    sig_width[const_base:const_base + n_consts] = const_width
    narrow1 = const_base + k0
    narrow8 = const_base + k0 + 1

    code = np.zeros(n_ops_total, np.uint8)
    width = np.zeros(n_ops_total, np.uint8)
    p0 = np.zeros(n_ops_total, np.uint8)
    p1 = np.zeros(n_ops_total, np.uint8)
    argv = np.zeros((n_ops_total, 3), np.int64)
    arity = np.zeros(n_ops_total, np.int64)

    next_op = 0
    if spec.counter_lfsr:
        cnt = reg_base + n_rand_regs
        lfsr = cnt + 1
        reg_width[n_rand_regs] = 32
        reg_width[n_rand_regs + 1] = 16
        sig_width[cnt], sig_width[lfsr] = 32, 16
        reg_init[n_rand_regs + 1] = 1
        one, taps = const_base + n_c + 2, const_base + n_c + 3

        def put(c, w, a, b=0, cc=0, q0=0, q1=0):
            nonlocal next_op
            k = next_op
            code[k], width[k], p0[k], p1[k] = c, w, q0, q1
            argv[k] = (a, b, cc)
            arity[k] = _ARITY[c]
            sig_width[op_base + k] = w
            next_op += 1
            return op_base + k

        cnt_next = put(OP["ADD"], 32, cnt, one)
        lsb = put(OP["BITS"], 1, lfsr, q0=0, q1=0)
        sh = put(OP["SHR"], 16, lfsr, q0=1)
        x = put(OP["XOR"], 16, sh, taps)
        lfsr_next = put(OP["MUX"], 16, lsb, x, sh)
        special_d = [cnt_next, lfsr_next]

    # layered random DAG
    layers = [np.arange(0, op_base, dtype=np.int64)]   # layer 0 = pool
    counts = np.full(spec.depth, spec.n_ops // spec.depth, np.int64)
    counts[: spec.n_ops % spec.depth] += 1
    classes = list(spec.mix.keys())
    cprob = np.array([spec.mix[c] for c in classes], np.float64)

    # memory read ops replace ordinary ops at random positions
    n_memrd = spec.n_mems * spec.mem_read_ports
    memrd_pos = set()
    if n_memrd:
        memrd_pos = set(int(x) for x in np.sort(rng.below(spec.n_ops, n_memrd)))
        while len(memrd_pos) < n_memrd:
            memrd_pos.add(int(rng.below(spec.n_ops, 1)[0]))
    memrd_list = sorted(memrd_pos)
    memrd_owner = {pos: j // spec.mem_read_ports for j, pos in enumerate(memrd_list)}

    def pick(L: int, n: int) -> np.ndarray:
        d = rng.geometric_half(n)
        src = np.maximum(L - d, 0)
        sizes = np.array([layers[s].size for s in range(L)], np.int64)
        idx = rng.below(sizes[src], n)
        out = np.empty(n, np.int64)
        for s in np.unique(src):
            m = src == s
            out[m] = layers[s][idx[m]]
        return out

    chained = np.zeros(n_signals, bool)   # chain members: exactly one reader
    dag_pos = 0
    for L in range(1, spec.depth + 1):
        k = int(counts[L - 1])
        cls = rng.choice(np.arange(len(classes)), cprob, k)
        c = np.zeros(k, np.int64)
        for ci, name in enumerate(classes):
            m = cls == ci
            if m.any():
                vals, pr = _SUB[name]
                c[m] = rng.choice(np.array(vals), pr, int(m.sum()))
        w = rng.choice(wv, wp, k)
        a = np.stack([pick(L, k), pick(L, k), pick(L, k)], axis=1)
        q0 = np.zeros(k, np.int64)
        q1 = np.zeros(k, np.int64)
        wa = sig_width[a[:, 0]]
        wb = sig_width[a[:, 1]]

        # MUL: both operands <= 32 bits
        m = (c == OP["MUL"]) & ((wa > 32) | (wb > 32))
        for _ in range(32):
            if not m.any():
                break
            n = int(m.sum())
            a[m, 0] = pick(L, n)
            a[m, 1] = pick(L, n)
            wa = sig_width[a[:, 0]]; wb = sig_width[a[:, 1]]
            m = (c == OP["MUL"]) & ((wa > 32) | (wb > 32))
        a[m & (wa > 32), 0] = narrow8
        a[m & (wb > 32), 1] = narrow8
        # CAT: w_a + w_b <= 64
        m = (c == OP["CAT"]) & (wa + wb > 64)
        for _ in range(32):
            if not m.any():
                break
            n = int(m.sum())
            a[m, 0] = pick(L, n)
            a[m, 1] = pick(L, n)
            wa = sig_width[a[:, 0]]; wb = sig_width[a[:, 1]]
            m = (c == OP["CAT"]) & (wa + wb > 64)
        a[m, 1] = narrow1
        wa = sig_width[a[:, 0]]; wb = sig_width[a[:, 1]]

        cmpm = np.isin(c, [OP["EQ"], OP["NEQ"], OP["LT"], OP["LEQ"], OP["GT"], OP["GEQ"],
                           OP["ANDR"], OP["ORR"], OP["XORR"]])
        w[cmpm] = 1
        m = c == OP["CAT"]
        w[m] = wa[m] + wb[m]
        q0[m] = wb[m]
        m = c == OP["BITS"]
        if m.any():
            n = int(m.sum())
            lo = rng.below(wa[m], n)
            hi = lo + rng.below(wa[m] - lo, n)
            q0[m], q1[m] = hi, lo
            w[m] = hi - lo + 1
        m = c == OP["SHL"]
        if m.any():
            q0[m] = rng.below(w[m], int(m.sum()))
        m = c == OP["SHR"]
        if m.any():
            q0[m] = rng.below(wa[m], int(m.sum()))
        m = c == OP["ANDR"]
        q0[m] = wa[m]

        # memory reads placed in this layer
        if memrd_list:
            lo_pos, hi_pos = dag_pos, dag_pos + k
            for pos in memrd_list:
                if lo_pos <= pos < hi_pos:
                    j = pos - lo_pos
                    c[j] = OP["MEMRD"]
                    w[j] = 64
                    mi = memrd_owner[pos]
                    q0[j], q1[j] = mi & 0xFF, mi >> 8

        # mux chains (when/else chains): the false operand (O = 2) of some MUXes
        # is a MUX of layer L-1 that nothing else reads (it leaves the operand
        # pool, and register D / write-port draws skip it); the head is no wider
        if spec.mux_chain_frac > 0 and L > 1:
            prev = layers[L - 1]
            cand = prev[(prev >= op_base + (5 if spec.counter_lfsr else 0))
                        & (code[np.maximum(prev - op_base, 0)] == OP["MUX"])]
            cand = cand[~np.isin(cand, a)]
            m = np.flatnonzero((c == OP["MUX"]) & (rng.uniform(k) < spec.mux_chain_frac))
            n = min(m.size, cand.size, max(0, prev.size - 8))
            if n:
                cand = cand[np.argsort(rng.u64(cand.size), kind="stable")][:n]
                m = m[:n]
                a[m, 2] = cand
                w[m] = np.minimum(w[m], sig_width[cand])
                chained[cand] = True
                layers[L - 1] = prev[~chained[prev]]

        sl = slice(next_op, next_op + k)
        code[sl], width[sl], p0[sl], p1[sl] = c, w, q0, q1
        argv[sl] = a
        arity[sl] = _ARITY[c]
        ids = op_base + np.arange(next_op, next_op + k, dtype=np.int64)
        sig_width[ids] = w
        layers.append(ids)
        next_op += k
        dag_pos += k

    assert next_op == n_ops_total
    # CSR args
    argoff = np.zeros(n_ops_total + 1, np.int64)
    argoff[1:] = np.cumsum(arity)
    sel = np.arange(3)[None, :] < arity[:, None]
    args = argv[sel]

    first_dag = op_base + (5 if spec.counter_lfsr else 0)
    reg_d = np.empty(n_regs, np.int64)
    reg_d[:n_rand_regs] = first_dag + rng.below(spec.n_ops, n_rand_regs)
    redraw = chained[reg_d[:n_rand_regs]]
    while redraw.any():
        reg_d[:n_rand_regs][redraw] = first_dag + rng.below(spec.n_ops, int(redraw.sum()))
        redraw = chained[reg_d[:n_rand_regs]]
    if spec.counter_lfsr:
        reg_d[n_rand_regs:] = special_d

    mem_words = np.full(spec.n_mems, spec.mem_words, np.uint32)
    mem_width = np.full(spec.n_mems, 64, np.uint8)
    nwp = spec.n_mems * spec.mem_write_ports
    wport = np.zeros((nwp, 4), np.int64)
    if nwp:
        wport[:, 0] = np.repeat(np.arange(spec.n_mems), spec.mem_write_ports)
        wport[:, 1:] = first_dag + rng.below(spec.n_ops, 3 * nwp).reshape(nwp, 3)
        redraw = chained[wport[:, 1:]]
        while redraw.any():
            wport[:, 1:][redraw] = first_dag + rng.below(spec.n_ops, int(redraw.sum()))
            redraw = chained[wport[:, 1:]]

    return Netlist(
        input_width=input_width.astype(np.uint8), reg_width=reg_width.astype(np.uint8),
        reg_d=reg_d.astype(np.uint32), reg_init=reg_init, const_width=const_width,
        const_value=const_value.astype(np.uint64), op_code=code, op_width=width,
        op_p0=p0, op_p1=p1, op_argoff=argoff.astype(np.uint32), args=args.astype(np.uint32),
        mem_words=mem_words, mem_width=mem_width, wport=wport.astype(np.uint32))


# ---------------------------------------------------------------------------
# Modular, enable-gated designs (low activity)
# ---------------------------------------------------------------------------
@dataclass
class ModularSpec:
    """M independent modules (each a random layered DAG of its own signals and
    primary inputs), a global 32-bit cycle counter, and per module an enable
    that is true one cycle in 2^k_m (k_m uniform in [k_lo, k_hi]): every
    register of module m loads its next state only when the enable is set,
    else holds -- the structure of clock-gated blocks in real designs.  Driven
    with inputs that change rarely (e.g. random values at reset, then held),
    a module's logic sees a change only in the cycle after its enable."""
    n_modules: int
    ops_per_module: int
    regs_per_module: int
    depth: int
    seed: int
    inputs_per_module: int = 16
    k_lo: int = 2
    k_hi: int = 7


def generate_modular(ms: ModularSpec) -> Netlist:
    rng = Rng(ms.seed, stream=0x40D00000 + GEN_VERSION)
    mods = [generate(DesignSpec(n_ops=ms.ops_per_module, n_regs=ms.regs_per_module, depth=ms.depth,
                                n_inputs=ms.inputs_per_module, seed=ms.seed * 1000 + m))
            for m in range(ms.n_modules)]
    M = ms.n_modules
    ks = ms.k_lo + rng.below(ms.k_hi - ms.k_lo + 1, M).astype(np.int64)
    phase = rng.below(1 << 20, M).astype(np.int64) & ((np.int64(1) << ks) - 1)

    def offs(v):
        return np.concatenate([[0], np.cumsum(v)]).astype(np.int64)
    in_off = offs([m.n_inputs for m in mods])
    reg_off = offs([m.n_regs for m in mods])
    const_off = offs([m.n_consts for m in mods])
    op_off = offs([m.n_ops for m in mods])
    I = int(in_off[-1])
    R = int(reg_off[-1]) + 1                   # + the cycle counter (last register)
    C = int(const_off[-1]) + 1 + M             # + const 1, + one phase constant per module
    reg_base, const_base = I, I + R
    op_base = I + R + C
    cnt = reg_base + R - 1
    c_one = const_base + int(const_off[-1])

    def remap(m, x):
        nl = mods[m]
        x = np.asarray(x, np.int64)
        return np.select(
            [x < nl.reg_base, x < nl.const_base, x < nl.op_base],
            [in_off[m] + x, reg_base + reg_off[m] + (x - nl.reg_base),
             const_base + const_off[m] + (x - nl.const_base)],
            op_base + op_off[m] + (x - nl.op_base))

    # enable logic and hold muxes, appended after every module op
    base_extra = op_base + int(op_off[-1])
    n_extra = 1 + 2 * M + (R - 1)
    e_code = np.zeros(n_extra, np.uint8)
    e_w = np.zeros(n_extra, np.uint8)
    e_p0 = np.zeros(n_extra, np.uint8)
    e_args = np.zeros((n_extra, 3), np.int64)
    e_ar = np.zeros(n_extra, np.int64)
    e_code[0], e_w[0], e_args[0, :2], e_ar[0] = OP["ADD"], 32, (cnt, c_one), 2
    for m in range(M):
        j = 1 + 2 * m
        e_code[j], e_w[j], e_p0[j], e_args[j, 0], e_ar[j] = OP["BITS"], 8, ks[m] - 1, cnt, 1
        e_code[j + 1], e_w[j + 1], e_ar[j + 1] = OP["EQ"], 1, 2
        e_args[j + 1, :2] = (base_extra + j, c_one + 1 + m)
    new_d = []
    j = 1 + 2 * M
    for m, nl in enumerate(mods):
        nr = nl.n_regs
        sl = slice(j, j + nr)
        e_code[sl], e_w[sl], e_ar[sl] = OP["MUX"], nl.reg_width, 3
        e_args[sl, 0] = base_extra + 2 + 2 * m                          # enable of module m
        e_args[sl, 1] = remap(m, nl.reg_d)                              # next state
        e_args[sl, 2] = reg_base + reg_off[m] + np.arange(nr)           # hold
        new_d.append(base_extra + np.arange(j, j + nr))
        j += nr
    e_flat = e_args[np.arange(3)[None, :] < e_ar[:, None]]

    args = np.concatenate([remap(m, nl.args) for m, nl in enumerate(mods)] + [e_flat])
    arity = np.concatenate([np.diff(nl.op_argoff.astype(np.int64)) for nl in mods] + [e_ar])
    argoff = np.concatenate([[0], np.cumsum(arity)])
    cat = np.concatenate
    return Netlist(
        input_width=cat([nl.input_width for nl in mods]).astype(np.uint8),
        reg_width=cat([nl.reg_width for nl in mods] + [np.array([32])]).astype(np.uint8),
        reg_d=cat(new_d + [np.array([base_extra])]).astype(np.uint32),
        reg_init=cat([nl.reg_init for nl in mods] + [np.zeros(1, np.uint64)]).astype(np.uint64),
        const_width=cat([nl.const_width for nl in mods] + [np.array([32] + [8] * M)]).astype(np.uint8),
        const_value=cat([nl.const_value for nl in mods] + [np.array([1] + list(phase), np.uint64)]).astype(np.uint64),
        op_code=cat([nl.op_code for nl in mods] + [e_code]).astype(np.uint8),
        op_width=cat([nl.op_width for nl in mods] + [e_w]).astype(np.uint8),
        op_p0=cat([nl.op_p0 for nl in mods] + [e_p0]).astype(np.uint8),
        op_p1=cat([nl.op_p1 for nl in mods] + [np.zeros(n_extra, np.uint8)]).astype(np.uint8),
        op_argoff=argoff.astype(np.uint32),
        args=args.astype(np.uint32))


def spec_quiet(seed: int = 6) -> ModularSpec:
    """1M ops in 64 enable-gated modules of 15,625 ops, depth 80, 1,024 registers
    and 16 inputs each."""
    return ModularSpec(n_modules=64, ops_per_module=15_625, regs_per_module=1024, depth=80, seed=seed)


# ---------------------------------------------------------------------------
# Stimulus seeds and per-instance cycle budgets
# ---------------------------------------------------------------------------
def xorshift_seeds(seed: int, n_inputs: int, n_instances: int) -> np.ndarray:
    """Initial xorshift64 states, uint64 [n_inputs][n_instances], never zero."""
    s = Rng(seed, stream=0x57140000).u64(n_inputs * n_instances).reshape(n_inputs, n_instances)
    s[s == 0] = np.uint64(0x9E3779B97F4A7C15)
    return s


def stimulus_values(seed: int, n_cycles: int, n_inputs: int, n_instances: int) -> np.ndarray:
    """Explicit per-cycle input values, uint64 [n_cycles][n_inputs][n_instances] (unmasked)."""
    return Rng(seed, stream=0x57150000).u64(n_cycles * n_inputs * n_instances).reshape(
        n_cycles, n_inputs, n_instances)


def cycle_budgets(seed: int, n_instances: int, lo: int = 1000, hi: int = 100_000) -> np.ndarray:
    """Per-instance cycle counts, uniform integers in [lo, hi]."""
    return (lo + Rng(seed, stream=0xC1C10000).below(hi - lo + 1, n_instances)).astype(np.uint32)

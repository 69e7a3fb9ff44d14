"""Closed-form pins for whole-cycle simulation in the oracle (CPU only).

Each circuit's expected behaviour comes from mathematics, not from another
simulator: modular counting, GF(2) matrix powers for the LFSR and the
xorshift64 stimulus, big-integer sums and products, fixed delays, a dict model
of a register file, prefix sums (Alg. 1 of the paper), and the paper's own
single-multiply example (Sec. 4.1).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import OP, Builder

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gf2_pow(M, n):
    R = np.eye(M.shape[0], dtype=np.int64)
    B = M.copy()
    while n:
        if n & 1:
            R = (R @ B) % 2
        B = (B @ B) % 2
        n >>= 1
    return R


def bits(x, w):
    return np.array([(x >> i) & 1 for i in range(w)], np.int64)


def from_bits(v):
    return int(sum(int(b) << i for i, b in enumerate(v)))


def shift_matrix(k, w=64):
    """Matrix of x -> x << k (k > 0) or x >> -k over GF(2)^w."""
    M = np.zeros((w, w), np.int64)
    for j in range(w):
        i = j + k
        if 0 <= i < w:
            M[i, j] = 1
    return M


def run(nl, cycles, n_inst=1, reset_first=True, **kw):
    sim = oracle.OracleSim(nl.to_bytes(), n_inst)
    if reset_first:
        sim.step(1, reset=True)
    out = sim.step(cycles, **kw)
    return sim, out


# ---------------------------------------------------------------- counter
@pytest.mark.parametrize("w,n", [(32, 10_000), (8, 1000), (16, 70_000), (1, 7)])
def test_counter_closed_form(w, n):
    b = Builder()
    q = b.reg(w)
    one = b.const(w, 1)
    b.connect(q, b.op("ADD", w, q, one))
    nl = b.build()
    sim, _ = run(nl, n)
    assert int(sim.vals[0, nl.reg_base]) == n % (1 << w)


# ---------------------------------------------------------------- LFSR
def lfsr_netlist():
    b = Builder()
    s = b.reg(16, init=1)
    taps = b.const(16, 0xB400)
    lsb = b.op("BITS", 1, s, p0=0, p1=0)
    sh = b.op("SHR", 16, s, p0=1)
    x = b.op("XOR", 16, sh, taps)
    b.connect(s, b.op("MUX", 16, lsb, x, sh))
    return b.build()


def lfsr_matrix():
    M = np.zeros((16, 16), np.int64)
    for j in range(16):
        img = (0xB400 if j == 0 else 0) ^ ((1 << j) >> 1)
        M[:, j] = bits(img, 16)
    return M


def test_lfsr_matrix_is_maximal():
    """Order of the step matrix is exactly 2^16 - 1 = 3*5*17*257 (primitive polynomial)."""
    M = lfsr_matrix()
    I = np.eye(16, dtype=np.int64)
    assert np.array_equal(gf2_pow(M, 65535), I)
    for p in [3, 5, 17, 257]:
        assert not np.array_equal(gf2_pow(M, 65535 // p), I)


def test_lfsr_golden_values():
    golden = {}
    for line in open(os.path.join(GOLDEN, "lfsr_b400.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, v = line.split()
        golden[int(n)] = int(v, 16)
    nl = lfsr_netlist()
    sim = oracle.OracleSim(nl.to_bytes(), 1)
    sim.step(1, reset=True)
    done = 0
    for n in sorted(golden):
        sim.step(n - done)
        done = n
        assert int(sim.vals[0, nl.reg_base]) == golden[n], n


def test_lfsr_period_and_never_zero():
    nl = lfsr_netlist()
    sim = oracle.OracleSim(nl.to_bytes(), 1)
    sim.step(1, reset=True)
    tr = sim.step(65535, probes=[nl.reg_base], probe_cycles=65535)[:, 0, 0]
    assert (tr != 0).all()
    assert tr[-1] == 1 and not (tr[:-1] == 1).any()          # first return to 1 at 65535
    assert len(np.unique(tr)) == 65535                        # visits every nonzero state


# ---------------------------------------------------------------- xorshift64 stimulus
def xorshift_matrix():
    I = np.eye(64, dtype=np.int64)
    A = (I + shift_matrix(13)) % 2          # x ^= x << 13
    B = (I + shift_matrix(-7)) % 2          # x ^= x >> 7
    C = (I + shift_matrix(17)) % 2          # x ^= x << 17
    return (C @ B @ A) % 2


def test_xorshift_triple_full_period():
    """Marsaglia's (13, 7, 17) step matrix has order 2^64 - 1."""
    T = xorshift_matrix()
    I = np.eye(64, dtype=np.int64)
    n = 2**64 - 1
    assert np.array_equal(gf2_pow(T, n), I)
    for p in [3, 5, 17, 257, 641, 65537, 6700417]:
        assert not np.array_equal(gf2_pow(T, n // p), I)


def test_xorshift_stimulus_matches_matrix_power():
    b = Builder()
    x = b.input(64)
    y = b.input(5)
    r = b.reg(1)
    b.connect(r, b.op("ORR", 1, x))
    nl = b.build()
    seeds = np.array([[0x0123456789ABCDEF, 1], [0xDEADBEEF, 0x8000000000000000]], np.uint64)
    sim = oracle.OracleSim(nl.to_bytes(), 2)
    xs = seeds.copy()
    tr = sim.step(50, mode=oracle.STIM_XORSHIFT, xs=xs, probes=[0, 1], probe_cycles=50)
    T = xorshift_matrix()
    for inst in range(2):
        for j, w in [(0, 64), (1, 5)]:
            s0 = bits(int(seeds[j, inst]), 64)
            for c in [0, 1, 2, 10, 49]:
                exp = from_bits(gf2_pow(T, c + 1) @ s0 % 2)
                assert int(tr[c, j, inst]) == exp % (1 << w)
            assert int(xs[j, inst]) == from_bits(gf2_pow(T, 50) @ s0 % 2)


# ---------------------------------------------------------------- trees and delays
def test_adder_and_multiplier_trees():
    b = Builder()
    ins = [b.input(16) for _ in range(8)]
    lvl = ins
    while len(lvl) > 1:
        lvl = [b.op("ADD", 32, lvl[i], lvl[i + 1]) for i in range(0, len(lvl), 2)]
    add_root = lvl[0]
    m = [b.op("MUL", 32, ins[0], ins[1]), b.op("MUL", 32, ins[2], ins[3])]
    mul_root = b.op("MUL", 64, m[0], m[1])
    mul_root8 = b.op("MUL", 8, m[0], m[1])
    sub = b.op("SUB", 32, ins[4], ins[5])
    r = b.reg(1)
    b.connect(r, b.op("XORR", 1, add_root))
    nl = b.build()
    n_inst = 64
    rng = np.random.default_rng(7)
    buf = rng.integers(0, 1 << 16, size=(3, 8, n_inst), dtype=np.uint64)
    buf[0, :, 0] = 0xFFFF
    sim, _ = run(nl, 3, n_inst, mode=oracle.STIM_BUFFER, buf=buf)
    vals = sim.read()
    last = buf[2]
    for i in range(n_inst):
        v = [int(t) for t in last[:, i]]
        assert int(vals[b.sid(add_root), i]) == sum(v) % 2**32
        prod = v[0] * v[1] % 2**32 * (v[2] * v[3] % 2**32)
        assert int(vals[b.sid(mul_root), i]) == prod % 2**64
        assert int(vals[b.sid(mul_root8), i]) == prod % 2**8
        assert int(vals[b.sid(sub), i]) == (v[4] - v[5]) % 2**32


@pytest.mark.parametrize("k", [1, 2, 5])
def test_shift_register_delay(k):
    """Registers whose D is another register's Q: Q_j(c) = in(c - j + 1)."""
    b = Builder()
    x = b.input(8)
    regs = [b.reg(8) for _ in range(k)]
    b.connect(regs[0], x)
    for j in range(1, k):
        b.connect(regs[j], regs[j - 1])
    b.connect(b.reg(1), b.op("NOT", 1, regs[-1]))
    nl = b.build()
    n = 20
    buf = np.arange(1, n + 1, dtype=np.uint64).reshape(n, 1, 1) * 7 % 251
    sim, tr = run(nl, n, mode=oracle.STIM_BUFFER, buf=buf,
                  probes=[b.sid(r) for r in regs], probe_cycles=n)
    for c in range(n):
        for j in range(k):
            exp = int(buf[c - j, 0, 0]) if c - j >= 0 else 0
            assert int(tr[c, j, 0]) == exp, (c, j)


def test_register_file_matches_dict_model():
    b = Builder()
    en, waddr, wdata, raddr = b.input(1), b.input(4), b.input(16), b.input(4)
    m = b.mem(8, width=12)
    rd = b.op("MEMRD", 12, raddr, p0=m)
    b.write_port(m, en, waddr, wdata)
    b.connect(b.reg(12), rd)
    nl = b.build()
    n = 200
    rng = np.random.default_rng(3)
    buf = np.stack([rng.integers(0, 2, n), rng.integers(0, 16, n), rng.integers(0, 1 << 16, n),
                    rng.integers(0, 16, n)], axis=1).astype(np.uint64).reshape(n, 4, 1)
    sim, tr = run(nl, n, mode=oracle.STIM_BUFFER, buf=buf, probes=[b.sid(rd)], probe_cycles=n)
    model = {}
    for c in range(n):
        e, wa, wd, ra = (int(t) for t in buf[c, :, 0])
        assert int(tr[c, 0, 0]) == model.get(ra % 8, 0), c      # read sees pre-edge data
        if e:
            model[wa % 8] = wd % (1 << 12)
    assert [int(t) for t in sim.read_mem()[:, 0]] == [model.get(a, 0) for a in range(8)]


def test_two_write_ports_higher_index_wins():
    b = Builder()
    a = b.input(3)
    m = b.mem(8)
    one = b.const(1, 1)
    v1, v2 = b.const(64, 111), b.const(64, 222)
    b.write_port(m, one, a, v1)
    b.write_port(m, one, a, v2)
    b.connect(b.reg(64), b.op("MEMRD", 64, a, p0=m))
    nl = b.build()
    buf = np.array([5], np.uint64).reshape(1, 1, 1)
    sim, _ = run(nl, 1, mode=oracle.STIM_BUFFER, buf=buf)
    assert int(sim.read_mem()[5, 0]) == 222


# ---------------------------------------------------------------- paper examples
def test_paper_single_multiply():
    """Sec. 4.1: LI = (1, 2, 4), the mask selects r = 0 and r = 2, LO = 4."""
    g = {}
    for line in open(os.path.join(GOLDEN, "paper_single_multiply.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        g[k] = [int(t) for t in v]
    b = Builder()
    regs = [b.reg(8, init=x) for x in g["LI"]]
    for r in regs:
        b.connect(r, r)
    prod = b.op("MUL", 8, regs[g["OIM_r"][0]], regs[g["OIM_r"][1]])
    nl = b.build()
    sim, _ = run(nl, 1)
    assert int(sim.vals[0, b.sid(prod)]) == g["LO"][0]


def test_paper_prefix_sum_iterative_rank():
    """Alg. 1: S_{i+1} = S_i + A_i with S_0 = 0, the iterative rank run as cycles."""
    b = Builder()
    a = b.input(16)
    s = b.reg(32)
    b.connect(s, b.op("ADD", 32, s, a))
    nl = b.build()
    A = np.array([3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5, 65535, 65535], np.uint64)
    sim, tr = run(nl, A.size, mode=oracle.STIM_BUFFER, buf=A.reshape(-1, 1, 1),
                  probes=[nl.reg_base], probe_cycles=A.size)
    assert [int(t) for t in tr[:, 0, 0]] == [int(x) for x in np.cumsum(A.astype(np.int64))]


def test_paper_dot_product():
    """Fig. dot: Z = sum_m A_m * B_m (map x, reduce +) as a multiply / add tree."""
    b = Builder()
    A = [b.input(8) for _ in range(4)]
    B = [b.input(8) for _ in range(4)]
    p = [b.op("MUL", 16, A[m], B[m]) for m in range(4)]
    z = b.op("ADD", 18, p[0], p[1], p[2], p[3])            # variadic reduce in O order
    b.connect(b.reg(18), z)
    nl = b.build()
    rng = np.random.default_rng(11)
    n_inst = 100
    buf = rng.integers(0, 256, size=(1, 8, n_inst), dtype=np.uint64)
    sim, _ = run(nl, 1, n_inst, mode=oracle.STIM_BUFFER, buf=buf)
    exp = (buf[0, :4].astype(np.int64) * buf[0, 4:].astype(np.int64)).sum(axis=0)
    assert np.array_equal(sim.read([b.sid(z)])[0].astype(np.int64), exp)


def test_reset_sets_init_and_counts_as_a_cycle():
    b = Builder()
    q = b.reg(8, init=42)
    b.connect(q, b.op("ADD", 8, q, b.const(8, 1)))
    nl = b.build()
    sim = oracle.OracleSim(nl.to_bytes(), 3)
    sim.step(5)
    assert (sim.vals[:, nl.reg_base] == 5).all()
    sim.step(1, reset=True)
    assert (sim.vals[:, nl.reg_base] == 42).all()
    sim.step(np.array([0, 1, 300], np.uint32))            # uneven cycle counts per instance
    assert [int(t) for t in sim.vals[:, nl.reg_base]] == [42, 43, (42 + 300) % 256]


def test_waveform_changes_of_counter_bits():
    """Bit k of a counter changes exactly at the cycles whose new value is a
    multiple of 2^k (closed form of a binary counter's toggling)."""
    from oracle.waveform import changes
    b = Builder()
    q = b.reg(8)
    b.connect(q, b.op("ADD", 8, q, b.const(8, 1)))
    bits = [b.op("BITS", 1, q, p0=k, p1=k) for k in range(4)]
    nl = b.build()
    sim = oracle.OracleSim(nl.to_bytes(), 1)
    sim.step(1, reset=True)
    probes = [b.sid(x) for x in bits]
    before = sim.read(probes)
    n = 40
    tr = sim.step(n, probes=probes, probe_cycles=n)
    ev = changes(before, tr, n)
    # the bits are combinational on Q: during cycle c (0-based) Q = c, and the
    # value recorded at the end of cycle c is bit k of c
    exp = []
    for c in range(n):
        for k in range(4):
            prev = ((c - 1) >> k) & 1 if c > 0 else 0
            if ((c >> k) & 1) != prev:
                exp.append((c, k, 0, (c >> k) & 1))
    assert [tuple(int(x) for x in r) for r in ev] == sorted(exp)
    assert sum(1 for r in ev if r[1] == 0) == n - 1          # bit 0 toggles every cycle after 0


def test_modular_generator_gates_registers_by_enable():
    """Generator pin for the low-activity workload: a register of module m takes
    a new value only in cycles whose counter value c has c mod 2^k_m = phase_m
    (its hold mux selects Q otherwise); the cycle counter counts cycles."""
    ms = synth.ModularSpec(n_modules=4, ops_per_module=300, regs_per_module=20, depth=6, seed=3,
                           inputs_per_module=4)
    nl = synth.generate_modular(ms)
    o = oracle.OracleSim(nl.to_bytes(), 4)
    xs = synth.xorshift_seeds(3, nl.n_inputs, 4)
    o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    cnt = nl.reg_base + nl.n_regs - 1
    # module m's enable is op (1 + 2m + 1) of the appended block; its BITS p0 = k - 1,
    # its phase constant is the EQ's second operand
    extra0 = nl.n_ops - (1 + 2 * ms.n_modules + (nl.n_regs - 1))
    ks, phases = [], []
    for m in range(ms.n_modules):
        bits = extra0 + 1 + 2 * m
        ks.append(int(nl.op_p0[bits]) + 1)
        phases.append(int(nl.const_value[int(nl.op_args(bits + 1)[1]) - nl.const_base]))
    prev = o.read()
    for c in range(40):
        q = int(o.read([cnt])[0, 0])
        assert q == c                                       # counter closed form
        o.step(1, mode=oracle.STIM_HOLD, xs=xs)
        cur = o.read()
        for m in range(ms.n_modules):
            regs = nl.reg_base + m * ms.regs_per_module + np.arange(ms.regs_per_module)
            if q % (1 << ks[m]) != phases[m]:
                assert np.array_equal(cur[regs], prev[regs]), (c, m)
        prev = cur


def _domain_counters(specs):
    """One 16-bit counter register (Q <- Q + 1) per (period, phase) domain, plus
    a base-clock counter."""
    b = Builder()
    one = b.const(16, 1)
    regs = []
    for per, ph in [(1, 0)] + list(specs):
        d = b.domain(per, ph)
        r = b.reg(16)
        b.connect(r, b.op("ADD", 16, r, one))
        b.clock(r, d)
        regs.append(r)
    return b.build(), [b.sid(r) for r in regs]


def test_clock_domains_count_their_ticks():
    """Multi-clock reading: a register of domain (p, f) loads only in cycles with
    (t + f) mod p == 0, t = non-reset cycles since reset; so a counter there holds
    #{t < n : (t + f) mod p == 0} after reset + n cycles (closed form)."""
    specs = [(2, 0), (2, 1), (4, 3), (8, 0), (16, 5)]
    nl, sig = _domain_counters(specs)
    o = oracle.OracleSim(nl.to_bytes(), 3)
    o.step(1, reset=True)
    done = 0
    for n in [1, 2, 5, 13, 40, 100]:
        o.step(n - done)
        done = n
        vals = o.read(sig)[:, 0]
        assert int(vals[0]) == n
        for (per, ph), v in zip(specs, vals[1:]):
            assert int(v) == sum(1 for t in range(n) if (t + ph) % per == 0), (per, ph, n)
    o.step(1, reset=True)                 # a reset restarts t
    o.step(3)
    vals = o.read(sig)[:, 0]
    assert [int(x) for x in vals] == [3] + [sum(1 for t in range(3) if (t + f) % p == 0) for p, f in specs]


def test_clock_domains_format_and_validation():
    nl, _ = _domain_counters([(4, 1)])
    assert synth.Netlist.from_bytes(nl.to_bytes()).to_bytes() == nl.to_bytes()
    bad = nl.to_bytes()
    # period 3 is not a power of two: the oracle refuses the netlist
    nl.dom_period = np.array([1, 3], np.uint32)
    with pytest.raises(ValueError):
        oracle.OracleSim(nl.to_bytes(), 1)
    assert oracle.OracleSim(bad, 1).n_regs == 2

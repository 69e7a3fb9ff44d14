"""The data-driven kernels' device code checked on the host (no GPU): the
library's own kernels.cuh (operand gathers of 1, 2, 4 or 8 packed lanes per
row class, the 32-bit narrow path, side-array operand lists, stimulus, clock
edge and write ports) and lower.cpp are compiled with the host compiler into
tests/layer_form_harness.cpp, which runs the LAYER form (and the TILE form's
lane tiles) phase by phase with every thread index of a phase called in turn.  Signals, memory words and
stimulus states must equal the oracle's for every lanes-per-thread width and
for thread counts equal to, above and below the number of lane chunks (the
fixed and the generic work mapping), over all lanes or tiles of lanes, with one,
two or four rows in flight per thread.  Planted mistakes in a temporary copy of
kernels.cuh must fail it.  The library runs these functions only on the GPU;
this checks their arithmetic and indexing without one."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from synth import Builder, DesignSpec

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(rt.__file__), "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
CUDA_INCLUDE = "/usr/local/cuda/include"
NP = 32                     # lanes (a power of two, as the library pads small batches)
P = ctypes.c_void_p


def build_harness(csrc: str, out_dir, opt: str = "-O1") -> ctypes.CDLL:
    so = os.path.join(str(out_dir), "harness.so")
    subprocess.run(["g++", "-std=c++17", opt, "-w", "-pthread", "-shared", "-fPIC", "-I", CUDA_INCLUDE, "-I", INCLUDE,
                    "-I", csrc, "-o", so, os.path.join(HERE, "layer_form_harness.cpp"),
                    os.path.join(csrc, "lower.cpp"), os.path.join(csrc, "inspect.cpp")], check=True)
    lib = ctypes.CDLL(so)
    lib.emu_create.restype = P
    lib.emu_create.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, P]
    lib.emu_step.argtypes = [P] + [ctypes.c_uint32] * 5 + [P, ctypes.c_int]
    lib.emu_read.argtypes = [P, ctypes.c_uint32, P]
    lib.emu_mem.restype = P
    lib.emu_mem.argtypes = [P]
    lib.emu_xs.restype = P
    lib.emu_xs.argtypes = [P]
    lib.emu_free.argtypes = [P]
    lib.emu_probe.argtypes = [P, P, ctypes.c_uint32, ctypes.c_int, P, ctypes.c_uint64, P]
    lib.emu_step_act.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int, ctypes.c_int, P]
    lib.emu_step_flow.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int]
    return lib


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("CUDA headers not found")
    return build_harness(CSRC, tmp_path_factory.mktemp("harness"))


def designs() -> dict:
    out = {}
    out["random+mem"] = (synth.generate(DesignSpec(n_ops=400, n_regs=30, depth=7, n_inputs=4, seed=3, n_mems=2,
                                                   mem_words=8, mem_write_ports=2,
                                                   input_widths=(8, 32, 1, 64))), False)
    chains = synth.generate(DesignSpec(n_ops=500, n_regs=30, depth=8, n_inputs=4, seed=71,
                                       input_widths=(8, 32, 1, 64), mux_chain_frac=0.7))
    out["chains"] = (chains, False)
    out["chains-fused"] = (chains, True)
    b = Builder()                                            # variadic folds, MUXCHAIN, ports
    ins = [b.input(w) for w in (64, 32, 8, 1, 1, 5)]
    m = b.mem(16, width=40)
    regs = [b.reg(w) for w in (64, 32, 40, 8)]
    ops = [b.op("ADD", 64, ins[0], ins[1], ins[2], regs[0], regs[1]),
           b.op("XOR", 32, ins[1], ins[2], regs[1], regs[3]),
           b.op("MUL", 64, ins[2], ins[5], regs[3], ins[2]),
           b.op("MUXCHAIN", 64, ins[3], ins[0], ins[4], regs[0], regs[3], ins[1], regs[2]),
           b.op("XORR", 1, regs[0]),
           b.op("MEMRD", 40, ins[5], p0=m)]
    t = b.op("CAT", 64, ops[5], b.op("BITS", 24, ops[0], p0=30, p1=7), p0=24)
    b.write_port(m, ins[3], ins[2], ops[0])
    b.write_port(m, ops[4], ins[5], ops[2])
    b.connect(regs[0], t)
    b.connect(regs[1], b.op("DSHR", 32, ops[1], ins[5]))
    b.connect(regs[2], ops[3])
    b.connect(regs[3], b.op("SUB", 8, ins[2], regs[3]))
    b.clock(regs[1], b.domain(4, 1))                         # and two clock domains
    b.clock(regs[3], b.domain(2, 0))
    out["wide+domains"] = (b.build(), False)
    out["counter+lfsr"] = (synth.generate(synth.spec_tiny(0)), False)
    b = Builder()                                            # no ops: edge copies only
    i0, k = b.input(8), b.const(16, 0xBEEF)
    r0, r1, r2 = b.reg(8, init=3), b.reg(16), b.reg(8)
    b.connect(r0, i0)
    b.connect(r1, k)
    b.connect(r2, r0)
    out["copies-only"] = (b.build(), False)
    out["byte results"] = (byte_results_design(), False)
    return out


def byte_results_design() -> synth.Netlist:
    """Ops with results of at most 8 bits (class-0 rows, the kernels' packed
    byte-lane form) over operands of every narrow class: each opcode at result
    widths 1, 4 and 8, once with operands of at most 8 bits and once with wider
    ones, shift amounts and bit ranges on both sides of a byte, two- and
    three-operand folds; registers feed results back so values change per cycle."""
    b = Builder()
    widths = (1, 3, 8, 12, 16, 24, 32)
    ins = [b.input(w) for w in widths]
    rw = (8, 5, 1, 16, 32, 7)
    regs = [b.reg(w, init=(37 * i + 11) & ((1 << w) - 1)) for i, w in enumerate(rw)]
    src = list(zip(ins + regs, widths + rw))
    small = [x for x, w in src if w <= 8]
    wide = [x for x, w in src if w > 8]
    k = 0

    def pick(pool, n):
        nonlocal k
        k += 1
        return [pool[(k * 3 + j * 5) % len(pool)] for j in range(n)]

    outs = []
    for w in (1, 4, 8):
        for pool in (small, wide, small + wide):
            for name, n in (("COPY", 1), ("AND", 2), ("OR", 2), ("XOR", 2), ("NOT", 1), ("ADD", 2),
                            ("SUB", 2), ("MUL", 2), ("DSHL", 2), ("DSHR", 2), ("EQ", 2), ("NEQ", 2),
                            ("LT", 2), ("LEQ", 2), ("GT", 2), ("GEQ", 2), ("MUX", 3), ("ORR", 1),
                            ("XORR", 1), ("AND", 3), ("XOR", 3), ("ADD", 3), ("OR", 3)):
                outs.append(b.op(name, w, *pick(pool, n)))
            for sh in (0, 1, 5, 7, 8, 9, 40):
                outs.append(b.op("SHL", w, *pick(pool, 1), p0=sh))
                outs.append(b.op("SHR", w, *pick(pool, 1), p0=sh))
                outs.append(b.op("CAT", w, *pick(pool, 2), p0=max(sh, 1)))
            for hi, lo in ((7, 0), (5, 2), (7, 7), (3, 0), (12, 9), (10, 3), (31, 8)):
                outs.append(b.op("BITS", w, *pick(pool, 1), p0=hi, p1=lo))
            for p0 in (1, 3, 8, 9, 16):
                outs.append(b.op("ANDR", w, *pick(pool, 1), p0=p0))
    # the ops' results feed the next cycle: byte results combined into each register
    for i, (r, wr) in enumerate(zip(regs, rw)):
        part = outs[i::len(regs)]
        acc = part[0]
        for x in part[1:]:
            acc = b.op("XOR", 8, acc, x)
        b.connect(r, b.op("ADD", wr, acc, *pick(wide, 1)))
    return b.build()


DESIGNS = designs()


def run_and_compare(lib, nl: synth.Netlist, fuse: bool, V: int, nthreads: int, U: int = 1, tile_lanes: int = 0,
                    seed: int = 1) -> None:
    nb = nl.to_bytes()
    xs = np.ascontiguousarray(synth.xorshift_seeds(seed, nl.n_inputs, NP))
    e = lib.emu_create(nb, len(nb), int(fuse), NP, xs.ctypes.data if nl.n_inputs else None)
    assert e
    orc = oracle.OracleSim(nb, NP)
    xo = xs.copy()
    rng = np.random.default_rng(seed)
    out = np.zeros(NP, np.uint64)
    try:
        for cycles, reset in [(1, True), (20, False), (None, False), (1, True), (7, False)]:
            budget = rng.integers(0, 12, NP).astype(np.uint32) if cycles is None else None
            ncyc = int(budget.max()) if budget is not None else cycles
            assert lib.emu_step(e, V, U, tile_lanes, nthreads, ncyc,
                                None if budget is None else budget.ctypes.data, int(reset)) == 0
            orc.step(budget if budget is not None else cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xo)
            for sig in range(nl.n_signals):
                if lib.emu_read(e, sig, out.ctypes.data) == 0:
                    assert np.array_equal(out, orc.vals[:, sig]), (sig, V, nthreads)
            words = orc.mem_total
            mem = np.ctypeslib.as_array(ctypes.cast(lib.emu_mem(e), ctypes.POINTER(ctypes.c_uint64)),
                                        (max(words, 1) * NP,))
            assert np.array_equal(mem[:words * NP].reshape(words, NP).T, orc.mems[:, :words])
            if nl.n_inputs:
                xk = np.ctypeslib.as_array(ctypes.cast(lib.emu_xs(e), ctypes.POINTER(ctypes.c_uint64)),
                                           (nl.n_inputs * NP,))
                assert np.array_equal(xk.reshape(nl.n_inputs, NP), xo)
    finally:
        lib.emu_free(e)


# (tile lanes (0: all lanes, the LAYER form), threads per phase as a function of
# the lane chunks of a span, rows in flight per thread)
MAPPINGS = {
    "one thread per chunk": (0, lambda ch: ch, 1),
    "more threads": (0, lambda ch: 3 * ch + 5, 1),
    "fewer threads": (0, lambda ch: max(1, ch // 3), 1),
    "all lanes, 4 rows in flight": (0, lambda ch: 2 * ch, 4),
    "tiles of 16 lanes, 2 rows in flight": (16, lambda ch: 5, 2),
    "tiles of 8 lanes, 4 rows in flight": (8, lambda ch: 3, 4),
}


@pytest.mark.parametrize("mapping", list(MAPPINGS))
@pytest.mark.parametrize("V", [1, 2, 4, 8])
@pytest.mark.parametrize("name", list(DESIGNS))
def test_layer_and_tile_forms_match_oracle(harness, name, V, mapping):
    nl, fuse = DESIGNS[name]
    tile, threads, U = MAPPINGS[mapping]
    run_and_compare(harness, nl, fuse, V, threads((tile or NP) // V), U=U, tile_lanes=tile)


@pytest.mark.parametrize("mapping", ["one thread per chunk", "fewer threads", "tiles of 8 lanes, 4 rows in flight"])
@pytest.mark.parametrize("V", [1, 4, 8])
def test_probes_every_cycle_and_change_records(harness, V, mapping):
    """Probes (Sec. 6.2 waveform generation): every cycle's values, and change
    records against the values at the start of the step, as the oracle's trace
    gives them."""
    from oracle.waveform import changes
    nl, fuse = DESIGNS["random+mem"]
    tile, threads, U = MAPPINGS[mapping]
    nthreads = threads((tile or NP) // V)
    nb = nl.to_bytes()
    xs = np.ascontiguousarray(synth.xorshift_seeds(5, nl.n_inputs, NP))
    e = harness.emu_create(nb, len(nb), 0, NP, xs.ctypes.data)
    orc, xo = oracle.OracleSim(nb, NP), xs.copy()
    probes = np.array([0, 3, nl.reg_base, nl.reg_base + 7, nl.op_base + 11, nl.op_base + 200, nl.n_signals - 1],
                      np.uint32)
    try:
        assert harness.emu_step(e, V, U, tile, nthreads, 1, None, 1) == 0
        orc.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xo)
        budgets = np.random.default_rng(V).integers(0, 15, NP).astype(np.uint32)
        ncyc = int(budgets.max())
        every = np.zeros((ncyc, probes.size, NP), np.uint64)
        assert harness.emu_probe(e, probes.ctypes.data, probes.size, 1, every.ctypes.data, 0, None) == 0
        assert harness.emu_step(e, V, U, tile, nthreads, ncyc, budgets.ctypes.data, 0) == 0
        tr = orc.step(budgets, mode=oracle.STIM_XORSHIFT, xs=xo, probes=probes, probe_cycles=ncyc)
        for i in range(NP):
            assert np.array_equal(every[:budgets[i], :, i], tr[:budgets[i], :, i]), i
        cap = 4096
        recs = np.zeros(3 * cap, np.uint64)
        count = np.zeros(1, np.uint64)
        assert harness.emu_probe(e, probes.ctypes.data, probes.size, 2, recs.ctypes.data, cap,
                                 count.ctypes.data) == 0
        before = orc.read(probes)
        assert harness.emu_step(e, V, U, tile, nthreads, 9, None, 0) == 0
        tr = orc.step(9, mode=oracle.STIM_XORSHIFT, xs=xo, probes=probes, probe_cycles=9)
        exp = changes(before, tr, 9)
        n = int(count[0])
        assert 0 < n == len(exp) <= cap
        r = recs[:3 * n].reshape(n, 3)
        got = np.stack([r[:, 0] & 0xFFFFFFFF, r[:, 0] >> 32, r[:, 1], r[:, 2]], axis=1).astype(np.uint64)
        got = got[np.lexsort(got.T[::-1])]
        assert np.array_equal(got, np.asarray(exp, np.uint64))
    finally:
        harness.emu_free(e)


KERNEL_MUTANTS = [
    ("narrow SUB operands swapped",
     "case OP_SUB: RT_LANES(a.x[v] - b.x[v]); break;\n    case OP_MUL: RT_LANES(a.x[v] * b.x[v]); if (ar == 3) RT_LANES(r.x[v] * c.x[v]); break;\n    case OP_SHL: RT_LANES(p0 >= 32u",
     "case OP_SUB: RT_LANES(b.x[v] - a.x[v]); break;\n    case OP_MUL: RT_LANES(a.x[v] * b.x[v]); if (ar == 3) RT_LANES(r.x[v] * c.x[v]); break;\n    case OP_SHL: RT_LANES(p0 >= 32u"),
    ("8-lane 1-byte gather: upper lanes from the lower word",
     "r.x[4 + v] = __byte_perm(t.y, 0u, 0x4440u + v);", "r.x[4 + v] = __byte_perm(t.x, 0u, 0x4440u + v);"),
    ("rows in flight: the next kind skips the rows past the boundary",
     "    return next;\n  }\n}", "    return r;\n  }\n}"),
    ("4-lane 2-byte store: lanes swapped within a word",
     "(uint32_t)(r.x[0] | (r.x[1] << 16)), (uint32_t)(r.x[2] | (r.x[3] << 16))",
     "(uint32_t)(r.x[1] | (r.x[0] << 16)), (uint32_t)(r.x[2] | (r.x[3] << 16))"),
    ("per-lane cycle budgets ignored",
     "return s.budget ? cyc < __ldg(&s.budget[lane]) : (lane < s.n_user && cyc < s.uniform);",
     "return lane < s.n_user && cyc < s.uniform;"),
    ("mux chain: the last set selector wins",
     "const bool take = (sel.x[v] & 1u) && !((done >> v) & 1u);", "const bool take = (sel.x[v] & 1u);"),
    ("reset ignores init values",
     "if (s.reset) {\n    const uint64_t init = __ldg(&d.reg_init[r]) & mk;",
     "if (s.reset) {\n    const uint64_t init = 0;"),
    ("register commit: the next register's table entries never advance",
     "        dsrc = dn;\n        qref = qn;", "        qref = qn;"),
    ("packed subtract: top bit of each byte not fixed up",
     "return ((a | H) - (b & ~H)) ^ ((a ^ ~b) & H);", "return ((a | H) - (b & ~H)) ^ ((a ^ b) & H);"),
    ("packed unsigned compare: the top bits ignored",
     "return ((x & b) | (~x & ~d)) & H;", "return ~d & H;"),
    ("packed shift left: bits crossing into the next byte kept",
     "return s >= 8u ? (T)0 : (a << s) & rep8<T>(0xFFu << s);", "return s >= 8u ? (T)0 : (a << s);"),
    ("packed parity: one fold dropped",
     "own bits only\n      x ^= x >> 2;", "own bits only\n"),
    ("8-lane 2-byte operand cut to its high bytes",
     "return (uint64_t)__byte_perm(t.x, t.y, 0x6420u) | ((uint64_t)__byte_perm(t.z, t.w, 0x6420u) << 32);",
     "return (uint64_t)__byte_perm(t.x, t.y, 0x7531u) | ((uint64_t)__byte_perm(t.z, t.w, 0x7531u) << 32);"),
    ("packed store of a partial mask writes every lane",
     "    if (m & (1u << v)) p[v] = (uint8_t)(r >> (8 * v));", "    p[v] = (uint8_t)(r >> (8 * v));"),
    ("packed form taken for a right shift of a wider operand",
     "return (dref >> 30) == 0u && (((PACK_LOW_OPS >> op) & 1u) || (bytes_in && ((PACK_BYTE_OPS >> op) & 1u)));",
     "return (dref >> 30) == 0u && (((PACK_LOW_OPS >> op) & 1u) || ((PACK_BYTE_OPS >> op) & 1u));"),
]


def test_planted_kernel_mistakes_are_caught(tmp_path):
    if not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("CUDA headers not found")
    with open(os.path.join(CSRC, "kernels.cuh")) as f:
        src = f.read()
    for k, (name, old, new) in enumerate(KERNEL_MUTANTS):
        assert src.count(old) == 1, "mutation site not found exactly once: " + name
        d = tmp_path / ("m%d" % k)
        d.mkdir()
        for f in ["lower.hpp", "lower.cpp", "inspect.cpp", "host_api.hpp", "flow_tables.hpp", "flow_items.cuh"]:
            shutil.copy(os.path.join(CSRC, f), str(d / f))
        (d / "kernels.cuh").write_text(src.replace(old, new))
        lib = build_harness(str(d), d, opt="-O0")   # quick to build; the runs are short
        caught = False
        for name_d in ["random+mem", "wide+domains", "chains-fused", "copies-only", "byte results"]:
            nl, fuse = DESIGNS[name_d]
            for V in (4, 8):
                try:
                    # rows in flight per thread: 4 for the mutant of that path
                    run_and_compare(lib, nl, fuse, V, NP // V, U=4 if "rows in flight" in name else 1)
                except AssertionError:
                    caught = True
                    break
            if caught:
                break
        assert caught, "no design catches: " + name


def run_activity(lib, V: int, hold: bool, np_: int = NP) -> tuple[int, int]:
    """Activity-aware evaluation on enable-gated modules against the oracle after
    every step (reset, quiet stretches, uneven budgets -- the next step's first
    cycle then evaluates everything -- and a second reset); returns the items
    evaluated and skipped."""
    nl = synth.generate_modular(synth.ModularSpec(n_modules=4, ops_per_module=150, regs_per_module=12, depth=6,
                                                  seed=9, inputs_per_module=4))
    nb = nl.to_bytes()
    xs = np.ascontiguousarray(synth.xorshift_seeds(9, nl.n_inputs, np_))
    e = lib.emu_create(nb, len(nb), 0, np_, xs.ctypes.data)
    orc, xo = oracle.OracleSim(nb, np_), xs.copy()
    counts = np.zeros(2, np.uint64)
    out = np.zeros(np_, np.uint64)
    rng = np.random.default_rng(V)
    try:
        for cycles, reset in [(1, True), (40, False), (None, False), (13, False), (1, True), (30, False)]:
            budget = rng.integers(0, 25, np_).astype(np.uint32) if cycles is None else None
            ncyc = int(budget.max()) if budget is not None else cycles
            mode = oracle.STIM_HOLD if hold and not reset else oracle.STIM_XORSHIFT
            assert lib.emu_step_act(e, V, ncyc, None if budget is None else budget.ctypes.data, int(reset),
                                    0 if mode == oracle.STIM_HOLD else 1, counts.ctypes.data) == 0
            orc.step(budget if budget is not None else cycles, reset=reset, mode=mode, xs=xo)
            for sig in range(nl.n_signals):
                if lib.emu_read(e, sig, out.ctypes.data) == 0:
                    assert np.array_equal(out, orc.vals[:, sig]), sig
    finally:
        lib.emu_free(e)
    return int(counts[0]), int(counts[1])


@pytest.mark.parametrize("V", [2, 4, 8])
@pytest.mark.parametrize("stimulus", ["held inputs", "random inputs"])
def test_activity_aware_evaluation(harness, V, stimulus):
    """Activity-aware evaluation (ops whose operands did not change in a 128-lane
    chunk are skipped there) equals the oracle; with held inputs most items are
    skipped."""
    evaluated, skipped = run_activity(harness, V, stimulus == "held inputs")
    assert evaluated > 0 and skipped > 0
    if stimulus == "held inputs":
        assert skipped > evaluated


@pytest.mark.parametrize("V", [1, 2, 8])
def test_activity_aware_evaluation_warp_cooperative(harness, V):
    """The warp-cooperative branch (a multiple of 32 lane chunks per row: 256
    lanes, two 128-lane stamp chunks): each warp's 32 threads run together,
    vote on hot rows and evaluate only those; equal to the oracle."""
    evaluated, skipped = run_activity(harness, V, True, np_=256)
    assert evaluated > 0 and skipped > evaluated


# (name, text, replacement, lanes per thread, lanes): 256 lanes at 8 per thread
# take the warp-cooperative branch with warps spanning two 128-lane stamp chunks
ACTIVITY_MUTANTS = [
    ("a row's third operand never makes it hot", "  if (ar >= 3) h |= hot_ref(m.z);\n", "\n", 4, NP),
    ("a register change left unstamped",
     "    *act_at(d, s, qref, lane) = (uint8_t)(s.act_g0 + cyc + 1u);\n", "\n", 4, NP),
    ("a warp checks only the first stamp chunk of its lanes",
     "const uint32_t ch_lo = first >> 7, ch_hi = (first + 32u * V - 1u) >> 7;",
     "const uint32_t ch_lo = first >> 7, ch_hi = ch_lo;", 8, 256),
]


def test_planted_activity_mistakes_are_caught(tmp_path):
    if not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("CUDA headers not found")
    with open(os.path.join(CSRC, "kernels.cuh")) as f:
        src = f.read()
    for k, (name, old, new, V, lanes) in enumerate(ACTIVITY_MUTANTS):
        assert src.count(old) == 1, "mutation site not found exactly once: " + name
        d = tmp_path / ("a%d" % k)
        d.mkdir()
        for f in ["lower.hpp", "lower.cpp", "inspect.cpp", "host_api.hpp", "flow_tables.hpp", "flow_items.cuh"]:
            shutil.copy(os.path.join(CSRC, f), str(d / f))
        (d / "kernels.cuh").write_text(src.replace(old, new))
        lib = build_harness(str(d), d, opt="-O0")   # quick to build; the runs are short
        with pytest.raises(AssertionError):
            run_activity(lib, V, True, np_=lanes)


def run_flow_and_compare(lib, nl: synth.Netlist, fuse: bool, n_warps: int, kw: int, np_: int = 4,
                         seed: int = 1) -> None:
    """The FLOW form's evaluation phase run by concurrent host threads (one per
    lane of each warp, waiting on one another's stamped words) over reset, even
    and uneven budgets and a second reset; every signal, memory word and
    stimulus state against the oracle after every step."""
    nb = nl.to_bytes()
    xs = np.ascontiguousarray(synth.xorshift_seeds(seed, nl.n_inputs, np_))
    e = lib.emu_create(nb, len(nb), int(fuse), np_, xs.ctypes.data if nl.n_inputs else None)
    assert e
    orc = oracle.OracleSim(nb, np_)
    xo = xs.copy()
    rng = np.random.default_rng(seed)
    out = np.zeros(np_, np.uint64)
    try:
        for cycles, reset in [(1, True), (9, False), (None, False), (1, True), (4, False)]:
            budget = rng.integers(0, 7, np_).astype(np.uint32) if cycles is None else None
            ncyc = int(budget.max()) if budget is not None else cycles
            assert lib.emu_step_flow(e, n_warps, kw, ncyc, None if budget is None else budget.ctypes.data,
                                     int(reset)) == 0
            orc.step(budget if budget is not None else cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xo)
            for sig in range(nl.n_signals):
                if lib.emu_read(e, sig, out.ctypes.data) == 0:
                    assert np.array_equal(out[:np_], orc.vals[:, sig]), (sig, n_warps, kw)
            words = orc.mem_total
            mem = np.ctypeslib.as_array(ctypes.cast(lib.emu_mem(e), ctypes.POINTER(ctypes.c_uint64)),
                                        (max(words, 1) * np_,))
            assert np.array_equal(mem[:words * np_].reshape(words, np_).T, orc.mems[:, :words])
    finally:
        lib.emu_free(e)


@pytest.mark.parametrize("n_warps,kw", [(1, 32), (2, 8), (3, 5)])
@pytest.mark.parametrize("name", ["random+mem", "chains-fused", "wide+domains", "byte results"])
def test_flow_form_matches_oracle(harness, name, n_warps, kw):
    nl, fuse = DESIGNS[name]
    run_flow_and_compare(harness, nl, fuse, n_warps, kw)


FLOW_MUTANTS = [
    ("an operand's high word dropped", "return (w.x & 0xFFFFFFFFull) | (w.y << 32);", "return w.x & 0xFFFFFFFFull;"),
    ("inputs, registers and constants copied without their high words",
     "st_relaxed_v2(flow_word(s, f, e.y, lane), v & 0xFFFFFFFFull, v >> 32);",
     "st_relaxed_v2(flow_word(s, f, e.y, lane), v & 0xFFFFFFFFull, 0ull);"),
    ("a result's high word stored without its value",
     "(r & 0xFFFFFFFFull) | sv, (r >> 32) | sv", "(r & 0xFFFFFFFFull) | sv, sv"),
]


def test_planted_flow_mistakes_are_caught(tmp_path):
    if not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("CUDA headers not found")
    with open(os.path.join(CSRC, "flow_items.cuh")) as f:
        src = f.read()
    for k, (name, old, new) in enumerate(FLOW_MUTANTS):
        assert src.count(old) == 1, "mutation site not found exactly once: " + name
        d = tmp_path / ("f%d" % k)
        d.mkdir()
        for f in ["lower.hpp", "lower.cpp", "inspect.cpp", "host_api.hpp", "flow_tables.hpp", "kernels.cuh"]:
            shutil.copy(os.path.join(CSRC, f), str(d / f))
        (d / "flow_items.cuh").write_text(src.replace(old, new))
        lib = build_harness(str(d), d, opt="-O0")
        nl, fuse = DESIGNS["wide+domains"]
        with pytest.raises(AssertionError):
            run_flow_and_compare(lib, nl, fuse, 1, 32)

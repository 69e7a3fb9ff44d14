"""The host-side lowering checks have teeth: plausible mistakes planted in a
temporary copy of the lowering (lower.cpp) -- swapped operand slots in the
descriptors, mux-chain fusion without its width condition, a clock-domain
enable of the wrong sense, an op placed on its operand's layer, write-port
enable and address swapped, an op's width field truncated -- each make the
round trip (the oracle on the decoded descriptors against the oracle on the
original netlist) fail.  The copy is compiled with the host compiler together
with the inspection unit into a temporary library; the library under test and
lower.cpp itself are never touched."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from synth import Builder, DesignSpec

CSRC = os.path.join(os.path.dirname(rt.__file__), "csrc")
INCLUDE = os.path.join(os.path.dirname(os.path.dirname(rt.__file__)), "include")
NONE = 0xFFFFFFFF

MUTANTS = [
    ("operand slots swapped in the descriptor",
     "      m.a = a[0];\n      m.b = a.size() > 1 ? a[1] : a[0];",
     "      m.a = a.size() > 1 ? a[1] : a[0];\n      m.b = a[0];"),
    ("fusion without the width condition",
     "return nl.code[k] == OP_MUX && fanout[sig] == 1 && nl.width[k] >= head_w;",
     "return nl.code[k] == OP_MUX && fanout[sig] == 1;"),
    ("clock-domain enable of the wrong sense",
     "enable[d] = put(OP_EQ, 1, {low, c_zero});", "enable[d] = put(OP_NEQ, 1, {low, c_zero});"),
    ("an op on its deepest operand's layer",
     "    level[opb + k] = lv + 1;", "    level[opb + k] = lv > 0 ? lv : 1;"),
    ("write-port enable and address swapped",
     "for (int t = 0; t < 3; t++) wp_lop[3ull * q + t] = edge_src(nl.wport[4ull * q + 1 + t]);",
     "for (int t = 0; t < 3; t++) wp_lop[3ull * q + t] = edge_src(nl.wport[4ull * q + 1 + (t < 2 ? 1 - t : t)]);"),
    ("width field truncated to 6 bits",
     "uint32_t ctl = code | (o.width << 8)", "uint32_t ctl = code | ((o.width & 63u) << 8)"),
]


def designs():
    """The designs every planted mistake is run on."""
    out = []
    b = Builder()                                            # variadic folds, chains, memory ports
    ins = [b.input(w) for w in (64, 32, 8, 1, 1, 5)]
    m = b.mem(16, width=40)
    regs = [b.reg(w) for w in (64, 32, 40, 8)]
    ops = [b.op("ADD", 64, ins[0], ins[1], ins[2], regs[0], regs[1]),
           b.op("SUB", 32, ins[1], regs[1]),
           b.op("MUL", 64, ins[2], ins[5], regs[3], ins[2]),
           b.op("MUXCHAIN", 64, ins[3], ins[0], ins[4], regs[0], regs[3], ins[1], regs[2]),
           b.op("LT", 1, ins[2], regs[3]),
           b.op("MEMRD", 40, ins[5], p0=m)]
    t = b.op("CAT", 64, ops[5], b.op("BITS", 24, ops[0], p0=30, p1=7), p0=24)
    b.write_port(m, ins[3], ins[2], ops[0])
    b.write_port(m, ops[4], ins[5], ops[2])
    b.connect(regs[0], t)
    b.connect(regs[1], ops[1])
    b.connect(regs[2], ops[3])
    b.connect(regs[3], b.op("XOR", 8, ops[4], regs[3], ins[2]))
    out.append((b.build(), False))
    b = Builder()                                            # a narrower inner mux under fusion
    s0, s1 = b.input(1), b.input(1)
    a, c, d = b.input(16), b.input(16), b.input(16)
    r = b.reg(16)
    b.connect(r, b.op("XOR", 16, b.op("MUX", 16, s0, a, b.op("MUX", 8, s1, c, d)), r))
    out.append((b.build(), True))
    nl = synth.generate(DesignSpec(n_ops=600, n_regs=40, depth=8, n_inputs=4, seed=81,
                                   input_widths=(8, 32, 1, 64), n_mems=2, mem_words=8))
    rng = np.random.default_rng(81)
    nl.dom_period = np.array([1, 2, 4, 8], np.uint32)      # clock domains
    nl.dom_phase = np.array([0, 1, 0, 5], np.uint32)
    nl.reg_domain = rng.integers(0, 4, nl.n_regs).astype(np.uint8)
    out.append((nl, False))
    return out


def _build(lower_src: str, tmp_path) -> ctypes.CDLL:
    src = tmp_path / "lower.cpp"
    src.write_text(lower_src)
    so = tmp_path / "libinspect.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-o", str(so),
                    str(src), os.path.join(CSRC, "inspect.cpp")], check=True)
    lib = ctypes.CDLL(str(so))
    lib.rteaal_design_lowered_netlist.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(rt.rteaal_load_opts),
                                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                                  ctypes.c_void_p, ctypes.c_uint64]
    lib.rteaal_last_error.restype = ctypes.c_char_p
    return lib


def _lowered(lib, nb: bytes, n_signals: int, fuse: bool):
    opts = rt.rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(fuse)
    n = ctypes.c_size_t()
    rc = lib.rteaal_design_lowered_netlist(nb, len(nb), ctypes.byref(opts), None, 0, ctypes.byref(n), None, 0)
    if rc:
        raise ValueError(lib.rteaal_last_error())
    out = ctypes.create_string_buffer(n.value)
    user2sig = np.zeros(n_signals, np.uint32)
    rc = lib.rteaal_design_lowered_netlist(nb, len(nb), ctypes.byref(opts), out, n.value, ctypes.byref(n),
                                           user2sig.ctypes.data, n_signals)
    if rc:
        raise ValueError(lib.rteaal_last_error())
    return out.raw[:n.value], user2sig


def _simulates_alike(lib, nl: synth.Netlist, fuse: bool, n: int = 16):
    nb = nl.to_bytes()
    low, user2sig = _lowered(lib, nb, nl.n_signals, fuse)
    keep = user2sig != NONE
    native, lowered = oracle.OracleSim(nb, n), oracle.OracleSim(low, n)
    xs = synth.xorshift_seeds(3, nl.n_inputs, n)
    xa, xb = xs.copy(), xs.copy()
    for cycles, reset in [(1, True), (20, False), (1, True), (9, False)]:
        native.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xa)
        lowered.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xb)
        assert np.array_equal(native.vals[:, keep], lowered.vals[:, user2sig[keep]])
        assert np.array_equal(native.mems[:, :native.mem_total], lowered.mems[:, :native.mem_total])


def _caught(lib) -> list:
    """The designs on which the round trip fails (an assertion, or a decoded
    netlist the oracle rejects)."""
    failed = []
    for i, (nl, fuse) in enumerate(designs()):
        try:
            _simulates_alike(lib, nl, fuse)
        except (AssertionError, ValueError):
            failed.append(i)
    return failed


def _source() -> str:
    with open(os.path.join(CSRC, "lower.cpp")) as f:
        return f.read()


def test_unchanged_copy_passes(tmp_path):
    assert _caught(_build(_source(), tmp_path)) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = _source()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    assert _caught(_build(src.replace(old, new), tmp_path)), "no design catches: " + name

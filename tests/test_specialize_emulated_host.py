"""The design-specialised kernel's arithmetic checked on the host (no GPU): the
CUDA source the generator writes for a design (rteaal_design_specialized_source)
is compiled with the host compiler behind a test-only shim that stands in for
the few CUDA built-ins it uses (the kernel qualifiers, the thread index, a
64-bit population count) and is called once per lane, exactly as one GPU
thread per lane would run it.  The rows and memory words it leaves must equal
the oracle's values after the same reset, cycles, uneven per-lane budgets and
second reset.  This tests the generator's text, not a CPU path of the library:
the library runs that kernel only on the GPU, where the GPU parity tests
compare it with the oracle as well."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import Builder, DesignSpec

NONE = 0xFFFFFFFF

SHIM = r'''
// Host stand-ins for the CUDA built-ins the generated kernel uses.
#define __global__
#define __launch_bounds__(n)
struct rt_index { unsigned x; };
static rt_index blockIdx, blockDim, threadIdx;
static inline int __popcll(unsigned long long v) { return __builtin_popcountll(v); }
#include "kernel.cu"
extern "C" void run_lanes(u8* st, u64* mem, u64* xs, const u64* stim, const u32* budget, const u32* reset_lane,
                          const u32* user_of_lane, u32 np, u32 n_user, u32 uniform, int stim_mode, int reset) {
  blockDim.x = 1;
  threadIdx.x = 0;
  for (u32 l = 0; l < np; l++) {
    blockIdx.x = l;
    rteaal_spec(st, mem, xs, stim, budget, reset_lane, user_of_lane, np, n_user, uniform, stim_mode, reset);
  }
}
'''


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()


def _compile(nb: bytes, fuse: bool, tmp_path) -> ctypes.CDLL:
    (tmp_path / "kernel.cu").write_text(rt.rteaal_design_specialized_source(nb, fuse_mux_chains=fuse))
    (tmp_path / "shim.cpp").write_text(SHIM)
    so = tmp_path / "spec.so"
    subprocess.run(["g++", "-std=c++17", "-O0", "-w", "-shared", "-fPIC", "-I", str(tmp_path), "-o", str(so),
                    str(tmp_path / "shim.cpp")], check=True)
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.run_lanes.argtypes = [P, P, P, P, P, P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_int, ctypes.c_int]
    return lib


def emulate_and_compare(nl: synth.Netlist, tmp_path, fuse: bool = False, n: int = 8, seed: int = 1):
    nb = nl.to_bytes()
    lib = _compile(nb, fuse, tmp_path)
    info, _ = rt.rteaal_design_lower(nb, fuse_mux_chains=fuse)
    low, user2sig = rt.rteaal_design_lowered_netlist(nb, nl.n_signals, fuse_mux_chains=fuse)
    refs = rt.rteaal_design_rows(nb, synth.Netlist.from_bytes(low).n_signals, fuse_mux_chains=fuse)
    st = np.zeros(info["state_bytes_per_lane"] * n, np.uint8)
    mem = np.zeros(max(info["mem_words_total"], 1) * n, np.uint64)
    xs = synth.xorshift_seeds(seed, nl.n_inputs, n)
    xk = np.ascontiguousarray(xs.copy()) if nl.n_inputs else np.zeros((1, n), np.uint64)
    orc = oracle.OracleSim(nb, n)
    xo = xs.copy()
    rng = np.random.default_rng(seed)

    def run(cycles, reset=False):
        budget = None
        if np.isscalar(cycles):
            uniform = int(cycles)
        else:
            budget = np.ascontiguousarray(cycles, np.uint32)
            uniform = 0
        lib.run_lanes(st.ctypes.data, mem.ctypes.data, xk.ctypes.data, None,
                      None if budget is None else budget.ctypes.data, None, None, n, n, uniform, 1, int(reset))
        orc.step(cycles, reset=reset, mode=oracle.STIM_XORSHIFT, xs=xo)
        check()

    def row(sig):
        ref = int(refs[user2sig[sig]])
        k, off = ref >> 30, ref & ((1 << 30) - 1)
        raw = st[off * n:off * n + (n << k)]
        return raw.view({0: np.uint8, 1: np.uint16, 2: np.uint32, 3: np.uint64}[k]).astype(np.uint64)

    consts = range(nl.n_inputs + nl.n_regs, nl.op_base)     # literals in the kernel, rows never written
    def check():
        for sig in range(nl.n_signals):
            if user2sig[sig] == NONE or sig in consts:
                continue
            assert np.array_equal(row(sig), orc.vals[:, sig]), sig
        words = orc.mem_total
        assert np.array_equal(mem[:words * n].reshape(words, n).T, orc.mems[:, :words])
        assert np.array_equal(xk[:nl.n_inputs], xo)

    run(1, reset=True)
    run(25)
    run(rng.integers(0, 20, n).astype(np.uint32))
    run(1, reset=True)
    run(9)


def test_random_design_with_memories(tmp_path):
    nl = synth.generate(DesignSpec(n_ops=400, n_regs=30, depth=7, n_inputs=4, seed=3, n_mems=2, mem_words=8,
                                   mem_write_ports=2, input_widths=(8, 32, 1, 64)))
    emulate_and_compare(nl, tmp_path)


def test_counter_lfsr_design(tmp_path):
    emulate_and_compare(synth.generate(synth.spec_tiny(0)), tmp_path, n=4)


@pytest.mark.parametrize("fuse", [False, True])
def test_mux_chains(fuse, tmp_path):
    nl = synth.generate(DesignSpec(n_ops=500, n_regs=30, depth=8, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7))
    emulate_and_compare(nl, tmp_path, fuse=fuse)


def test_wide_ops_memories_and_clock_domains(tmp_path):
    b = Builder()
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
    b.clock(regs[1], b.domain(4, 1))
    b.clock(regs[3], b.domain(2, 0))
    emulate_and_compare(b.build(), tmp_path, n=16)

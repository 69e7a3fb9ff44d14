"""Parity oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (``cpu_baseline`` and ``--impl reference``) may import this package.  The
product path (``paper_2601_18140_gb300``) never imports it and shares no code
with it.

Three independent evaluators live here:
  * ``oracle.c`` (via :class:`OracleSim`): gate-by-gate cycle simulation in
    topological order -- the plain definition of full-cycle RTL simulation
    (Sec. 2.1, Fig. 1).  Used for every parity comparison.
  * :mod:`oracle.pyeval`: a pure-Python evaluator with Python-int semantics,
    used for brute force on tiny circuits and per-opcode exhaustive checks.
  * :mod:`oracle.cascade`: the paper's Einsum cascade (Cascade 1, Sec. 4.2)
    written in its own order and notation (levelisation, explicit identity
    operations, OI / LO / LO_sel / LI_{i+1}), used to pin the cascade reading
    against the plain definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_lib = None

STIM_HOLD, STIM_XORSHIFT, STIM_BUFFER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into an in-tree shared library (gcc, portable flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u8p = ctypes.c_char_p
        P = ctypes.c_void_p
        L.oracle_sizes.argtypes = [u8p, ctypes.c_size_t, P]
        L.oracle_init.argtypes = [u8p, ctypes.c_size_t, ctypes.c_uint32, P, P]
        L.oracle_run.argtypes = [u8p, ctypes.c_size_t, ctypes.c_uint32, P, P, P, P, ctypes.c_int,
                                 ctypes.c_int, P, ctypes.c_uint32, P, ctypes.c_uint32,
                                 ctypes.c_uint32, P, ctypes.c_uint32, P, ctypes.c_uint32,
                                 ctypes.c_int]
        L.oracle_eval_one.argtypes = [ctypes.c_uint32] * 4 + [P, ctypes.c_uint32]
        L.oracle_eval_one.restype = ctypes.c_uint64
        L.oracle_eval_batch.argtypes = [ctypes.c_uint32] * 4 + [P, ctypes.c_uint32, ctypes.c_uint64, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def eval_one(code: int, width: int, operands, p0: int = 0, p1: int = 0) -> int:
    ops = np.ascontiguousarray(np.array(operands, dtype=np.uint64))
    return int(lib().oracle_eval_one(code, width, p0, p1, _ptr(ops), ops.size))


def eval_batch(code: int, width: int, operands: np.ndarray, p0: int = 0, p1: int = 0) -> np.ndarray:
    """Evaluate one operation type on many operand rows ([n][k] uint64)."""
    ops = np.ascontiguousarray(operands, dtype=np.uint64)
    out = np.zeros(ops.shape[0], np.uint64)
    lib().oracle_eval_batch(code, width, p0, p1, _ptr(ops), ops.shape[1], ops.shape[0], _ptr(out))
    return out


class OracleSim:
    """State of ``n_inst`` independent instances of one netlist, on the host."""

    def __init__(self, netlist: bytes, n_inst: int):
        self.nl = bytes(netlist)
        sizes = np.zeros(8, np.uint64)
        rc = lib().oracle_sizes(self.nl, len(self.nl), _ptr(sizes))
        if rc:
            raise ValueError("oracle: netlist format error")
        (self.n_signals, self.mem_total, self.n_inputs, self.n_regs, self.n_consts,
         self.n_ops, self.n_mems, self.n_wports) = (int(x) for x in sizes)
        self.n_inst = n_inst
        self.vals = np.zeros((n_inst, self.n_signals), np.uint64)
        self.mems = np.zeros((n_inst, max(self.mem_total, 1)), np.uint64)
        rc = lib().oracle_init(self.nl, len(self.nl), n_inst, _ptr(self.vals), _ptr(self.mems))
        assert rc == 0
        self.ticks = np.zeros(n_inst, np.uint32)   # non-reset cycles since reset (clock domains)

    def step(self, cycles, reset: bool = False, mode: int = STIM_HOLD, xs: np.ndarray | None = None,
             buf: np.ndarray | None = None, probes=None, probe_cycles: int = 0,
             threads: int = 1) -> np.ndarray | None:
        """Advance every instance.  ``cycles``: int or per-instance array.
        ``xs``: uint64 [n_inputs][n_inst] xorshift states, updated in place.
        ``buf``: uint64 [cycles][n_inputs][n_inst] explicit input values.
        ``probes``: signal ids; returns [probe_cycles][n_probes][n_inst]."""
        cyc = np.ascontiguousarray(np.broadcast_to(np.asarray(cycles, np.uint32), (self.n_inst,)))
        if xs is not None:
            assert xs.dtype == np.uint64 and xs.flags.c_contiguous and xs.shape == (self.n_inputs, self.n_inst)
        stim_cycles = 0
        if buf is not None:
            buf = np.ascontiguousarray(buf, dtype=np.uint64)
            assert buf.shape[1:] == (self.n_inputs, self.n_inst)
            stim_cycles = buf.shape[0]
        out = None
        psig = None
        if probes is not None:
            psig = np.ascontiguousarray(np.asarray(probes, np.uint32))
            out = np.zeros((probe_cycles, psig.size, self.n_inst), np.uint64)
        rc = lib().oracle_run(self.nl, len(self.nl), self.n_inst, _ptr(self.vals), _ptr(self.mems),
                              _ptr(self.ticks), _ptr(cyc), int(reset), mode, _ptr(xs), self.n_inst, _ptr(buf),
                              self.n_inst, stim_cycles, _ptr(psig),
                              0 if psig is None else psig.size, _ptr(out), probe_cycles, threads)
        if rc:
            raise ValueError("oracle_run failed: %d" % rc)
        return out

    def read(self, signals=None) -> np.ndarray:
        """Signal values, [n_signals][n_inst] (signal-major, like the device layout)."""
        if signals is None:
            return self.vals.T.copy()
        return self.vals[:, np.asarray(signals, np.int64)].T.copy()

    def read_mem(self) -> np.ndarray:
        """Memory words, [mem_words_total][n_inst]."""
        return self.mems[:, : self.mem_total].T.copy()

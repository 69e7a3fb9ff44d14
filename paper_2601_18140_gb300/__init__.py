"""Python binding of librteaal.so (include/rteaal.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels; this module
only converts Python / numpy / torch arguments to the C ABI.  There is no CPU
fallback: if the compiled library is missing, importing the binding's
functions raises.

PyTorch is used for device memory (its caching allocator is handed to the
library as the device-memory provider) and for streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librteaal.so")

RTEAAL_OK, RTEAAL_E_INVALID, RTEAAL_E_FORMAT, RTEAAL_E_NOMEM = 0, -1, -2, -3
RTEAAL_E_CUDA, RTEAAL_E_TIMEOUT, RTEAAL_E_BUSY, RTEAAL_E_UNSUPPORTED = -4, -5, -6, -7
RTEAAL_KERNEL_AUTO, RTEAAL_KERNEL_LAYER, RTEAAL_KERNEL_TILE = 0, 1, 2
RTEAAL_KERNEL_GRID, RTEAAL_KERNEL_LAYER_GRAPH, RTEAAL_KERNEL_STREAM = 3, 4, 5
RTEAAL_STIM_HOLD, RTEAAL_STIM_XORSHIFT, RTEAAL_STIM_BUFFER = 0, 1, 2
RTEAAL_PROBE_LAST, RTEAAL_PROBE_EVERY, RTEAAL_PROBE_CHANGES = 0, 1, 2
RTEAAL_STEP_RESET = 1

KERNELS = {"auto": 0, "layer": 1, "tile": 2, "grid": 3, "layer_graph": 4, "stream": 5, "specialized": 6,
           "cluster": 7, "flow": 8}


class RteaalError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("rteaal error %d: %s" % (code, msg))
        self.code = code


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_ALLOC_FN = ctypes.CFUNCTYPE(_P, ctypes.c_size_t, _P)
_FREE_FN = ctypes.CFUNCTYPE(None, _P, ctypes.c_size_t, _P)


class rteaal_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", _P)]


class rteaal_load_opts(ctypes.Structure):
    _fields_ = [("allocator", ctypes.POINTER(rteaal_allocator)), ("device", ctypes.c_int),
                ("fuse_mux_chains", ctypes.c_int)]


class rteaal_design_stats(ctypes.Structure):
    _fields_ = [(n, _U32) for n in ["n_signals", "n_inputs", "n_regs", "n_consts", "n_ops",
                                    "n_mems", "n_wports", "n_layers", "n_groups", "n_slots",
                                    "n_lowered_ops", "max_layer_ops"]] + \
               [(n, _U64) for n in ["op_operands", "mem_words_total", "metadata_bytes",
                                    "state_bytes_per_lane"]] + [("n_fused", _U32)]


class rteaal_sim_opts(ctypes.Structure):
    _fields_ = [("allocator", ctypes.POINTER(rteaal_allocator)),
                ("expected_cycles", ctypes.POINTER(_U32)),
                ("xorshift_seed", ctypes.POINTER(_U64)),
                ("kernel", ctypes.c_int), ("tile_lanes", _U32), ("threads", _U32),
                ("ctas_per_sm", _U32), ("unroll", _U32), ("lanes_per_thread", _U32),
                ("activity", ctypes.c_int), ("cluster_ctas", _U32), ("cluster_resident", ctypes.c_int)]


class rteaal_sim_stats(ctypes.Structure):
    _fields_ = [("n_instances", _U32), ("n_lanes", _U32), ("device_bytes", _U64),
                ("kernel", ctypes.c_int), ("tile_lanes", _U32), ("threads", _U32),
                ("ctas_per_sm", _U32), ("unroll", _U32), ("grid", _U32), ("lanes_per_thread", _U32),
                ("activity", ctypes.c_int), ("last_span", _U32), ("last_grid", _U32),
                ("cluster_ctas", _U32), ("cluster_resident", ctypes.c_int)]


class rteaal_tune_trial(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_lanes", _U32), ("threads", _U32),
                ("ctas_per_sm", _U32), ("unroll", _U32), ("grid", _U32), ("lanes_per_thread", _U32),
                ("ms", ctypes.c_float)]


class rteaal_cycles(ctypes.Structure):
    _fields_ = [("uniform", _U64), ("per_instance", ctypes.POINTER(_U32)),
                ("reset_per_instance", ctypes.POINTER(_U32))]


class rteaal_stimulus(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("values", _P), ("values_on_host", ctypes.c_int)]


class rteaal_probes(ctypes.Structure):
    _fields_ = [("signals", ctypes.POINTER(_U32)), ("n", _U32), ("mode", ctypes.c_int),
                ("out", _P), ("out_on_host", ctypes.c_int), ("capacity", _U64),
                ("count", ctypes.POINTER(_U64))]


CHANGE_DTYPE = np.dtype([("cycle", "<u4"), ("probe", "<u4"), ("instance", "<u4"), ("pad", "<u4"),
                         ("value", "<u8")])


EXPORTS = ["rteaal_design_load", "rteaal_design_info", "rteaal_design_free", "rteaal_sim_create",
           "rteaal_sim_info", "rteaal_sim_destroy", "rteaal_sim_configure", "rteaal_sim_autotune", "rteaal_sim_footprint", "rteaal_step",
           "rteaal_sync", "rteaal_state_read", "rteaal_state_write", "rteaal_mem_read",
           "rteaal_mem_write", "rteaal_stim_state_read", "rteaal_stim_state_write",
           "rteaal_last_error", "rteaal_step_static", "rteaal_sim_reset_lanes",
           "rteaal_design_signals", "rteaal_sim_activity", "rteaal_design_specialize",
           "rteaal_design_lower", "rteaal_design_specialize_host", "rteaal_design_single_clock",
           "rteaal_design_lowered_netlist", "rteaal_design_rows", "rteaal_design_flow_tables",
           "rteaal_design_specialized_source"]
STATIC_MAX_LANES = 65536

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librteaal.so is not built (run __graft_entry__.build() or "
                              "python paper_2601_18140_gb300/build.py); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.rteaal_last_error.restype = ctypes.c_char_p
        L.rteaal_design_load.argtypes = [ctypes.c_char_p, ctypes.c_size_t,
                                         ctypes.POINTER(rteaal_load_opts), ctypes.POINTER(_P)]
        L.rteaal_design_info.argtypes = [_P, ctypes.POINTER(rteaal_design_stats)]
        L.rteaal_design_specialize_host.argtypes = [ctypes.c_char_p, ctypes.c_size_t,
                                                    ctypes.POINTER(rteaal_load_opts), ctypes.POINTER(_U64),
                                                    ctypes.POINTER(_U64)]
        L.rteaal_design_lowered_netlist.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(rteaal_load_opts),
                                                    _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _P, _U64]
        L.rteaal_design_specialized_source.argtypes = [ctypes.c_char_p, ctypes.c_size_t,
                                                       ctypes.POINTER(rteaal_load_opts), _P, ctypes.c_size_t,
                                                       ctypes.POINTER(ctypes.c_size_t)]
        L.rteaal_design_rows.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(rteaal_load_opts), _P, _U64]
        L.rteaal_design_flow_tables.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(rteaal_load_opts),
                                                _P, ctypes.POINTER(_U64), _P, ctypes.POINTER(_U64), _P,
                                                ctypes.POINTER(_U64)]
        L.rteaal_design_single_clock.argtypes = [ctypes.c_char_p, ctypes.c_size_t, _P, ctypes.c_size_t,
                                                 ctypes.POINTER(ctypes.c_size_t), _P, _U64]
        L.rteaal_design_lower.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(rteaal_load_opts),
                                          ctypes.POINTER(rteaal_design_stats), _P, _U32]
        L.rteaal_design_free.argtypes = [_P]
        L.rteaal_design_specialize.argtypes = [_P, ctypes.POINTER(_U64)]
        L.rteaal_design_signals.argtypes = [_P, _P, _U64]
        L.rteaal_sim_create.argtypes = [_P, _U32, ctypes.POINTER(rteaal_sim_opts), ctypes.POINTER(_P)]
        L.rteaal_sim_info.argtypes = [_P, ctypes.POINTER(rteaal_sim_stats)]
        L.rteaal_sim_destroy.argtypes = [_P]
        L.rteaal_sim_destroy.restype = None
        L.rteaal_sim_configure.argtypes = [_P, ctypes.POINTER(rteaal_sim_opts)]
        L.rteaal_sim_autotune.argtypes = [_P, _U32, _U32, ctypes.POINTER(rteaal_tune_trial), _U32,
                                          ctypes.POINTER(_U32), _P]
        L.rteaal_sim_activity.argtypes = [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), _P]
        L.rteaal_sim_footprint.argtypes = [_P, _U32]
        L.rteaal_sim_footprint.restype = _U64
        L.rteaal_step.argtypes = [_P, ctypes.POINTER(rteaal_cycles), ctypes.POINTER(rteaal_stimulus),
                                  ctypes.POINTER(rteaal_probes), _U32, _P]
        L.rteaal_sync.argtypes = [_P, _P]
        L.rteaal_sim_reset_lanes.argtypes = [_P, _U32, _U32, _P, _P]
        for n in ["rteaal_state_read", "rteaal_state_write"]:
            getattr(L, n).argtypes = [_P, ctypes.POINTER(_U32), _U32, _U32, _U32, _P, _P]
        for n in ["rteaal_mem_read", "rteaal_mem_write", "rteaal_stim_state_read",
                  "rteaal_stim_state_write"]:
            getattr(L, n).argtypes = [_P, _U32, _U32, _P, _P]
        L.rteaal_step_static.argtypes = [_P, _P, _P, _P, _U32, ctypes.POINTER(_U32), _U32,
                                         ctypes.c_int, _U32, _P]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != RTEAAL_OK:
        raise RteaalError(rc, lib().rteaal_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray | None, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _dev_ptr(x) -> int | None:
    """Device (or pinned host) pointer of a torch tensor, or an int passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError("expected a torch tensor, numpy array or int pointer")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream) or None
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None


# ------------------------------------------------------------ torch allocator
_torch_alloc: rteaal_allocator | None = None


def torch_allocator() -> rteaal_allocator:
    """PyTorch's caching allocator as an rteaal_allocator (kept alive here)."""
    global _torch_alloc
    if _torch_alloc is None:
        import torch

        def _alloc(n, _ctx):
            try:
                dev = torch.cuda.current_device()
                return int(torch.cuda.caching_allocator_alloc(int(n), dev,
                                                              torch.cuda.current_stream(dev)))
            except Exception:
                return None

        def _free(p, _n, _ctx):
            torch.cuda.caching_allocator_delete(int(p))

        a = rteaal_allocator()
        a.alloc = _ALLOC_FN(_alloc)
        a.free = _FREE_FN(_free)
        a.ctx = None
        a._keep = (a.alloc, a.free)
        _torch_alloc = a
    return _torch_alloc


# ------------------------------------------------------------ C ABI, same names
def rteaal_design_load(netlist: bytes, opts: rteaal_load_opts | None = None) -> int:
    out = _P()
    _check(lib().rteaal_design_load(netlist, len(netlist),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(out)))
    return out.value


def rteaal_design_info(design: int) -> dict:
    st = rteaal_design_stats()
    _check(lib().rteaal_design_info(design, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in st._fields_}


def rteaal_design_lower(netlist: bytes, fuse_mux_chains: bool = False) -> tuple[dict, np.ndarray]:
    """The lowering on the host (no device): the design figures and the lowered
    op count of every layer."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    st = rteaal_design_stats()
    _check(lib().rteaal_design_lower(netlist, len(netlist), ctypes.byref(opts), ctypes.byref(st), None, 0))
    layer_ops = np.zeros(max(st.n_layers, 1), np.uint32)
    _check(lib().rteaal_design_lower(netlist, len(netlist), ctypes.byref(opts), ctypes.byref(st),
                                     layer_ops.ctypes.data, st.n_layers))
    return {n: getattr(st, n) for n, _ in st._fields_}, layer_ops[:st.n_layers]


def rteaal_design_single_clock(netlist: bytes, n_signals: int) -> tuple[bytes, np.ndarray]:
    """The one-clock netlist the library simulates (hidden cycle counter, enables
    and hold muxes for clock domains) and, per caller signal, its id there."""
    n = ctypes.c_size_t()
    _check(lib().rteaal_design_single_clock(netlist, len(netlist), None, 0, ctypes.byref(n), None, 0))
    out = ctypes.create_string_buffer(n.value)
    user2x = np.zeros(n_signals, np.uint32)
    _check(lib().rteaal_design_single_clock(netlist, len(netlist), out, n.value, ctypes.byref(n),
                                            user2x.ctypes.data, n_signals))
    return out.raw[:n.value], user2x


def rteaal_design_lowered_netlist(netlist: bytes, n_signals: int,
                                  fuse_mux_chains: bool = False) -> tuple[bytes, np.ndarray]:
    """The lowered design written back as a netlist (one signal per state row, one
    op per descriptor) and, per caller signal, its id there (0xFFFFFFFF: fused away)."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    n = ctypes.c_size_t()
    _check(lib().rteaal_design_lowered_netlist(netlist, len(netlist), ctypes.byref(opts), None, 0,
                                               ctypes.byref(n), None, 0))
    out = ctypes.create_string_buffer(n.value)
    user2sig = np.zeros(n_signals, np.uint32)
    _check(lib().rteaal_design_lowered_netlist(netlist, len(netlist), ctypes.byref(opts), out, n.value,
                                               ctypes.byref(n), user2sig.ctypes.data, n_signals))
    return out.raw[:n.value], user2sig


def rteaal_design_rows(netlist: bytes, n_rows: int, fuse_mux_chains: bool = False) -> np.ndarray:
    """Row reference (width class << 30 | per-lane byte offset) of every row of the
    lowered design, indexed like the signals of rteaal_design_lowered_netlist."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    refs = np.zeros(n_rows, np.uint32)
    _check(lib().rteaal_design_rows(netlist, len(netlist), ctypes.byref(opts), refs.ctypes.data, n_rows))
    return refs


def rteaal_design_flow_tables(netlist: bytes, fuse_mux_chains: bool = False):
    """The FLOW form's tables of the lowered design (host only): op [n_ops][8]
    (operand rows a, b, c with bit 31 on rows written in the cycle, output row,
    ctl, output reference, side-array offset, operand count), ext [n_ext]
    (flagged operand rows of ops with more than three operands) and pool
    [n_pool][2] ({reference, row} of inputs, registers, constants)."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    n_op, n_ext, n_pool = _U64(0), _U64(0), _U64(0)
    _check(lib().rteaal_design_flow_tables(netlist, len(netlist), ctypes.byref(opts), None, ctypes.byref(n_op),
                                           None, ctypes.byref(n_ext), None, ctypes.byref(n_pool)))
    op = np.zeros((n_op.value, 8), np.uint32)
    ext = np.zeros(n_ext.value, np.uint32)
    pool = np.zeros((n_pool.value, 2), np.uint32)
    _check(lib().rteaal_design_flow_tables(netlist, len(netlist), ctypes.byref(opts), op.ctypes.data,
                                           ctypes.byref(n_op), ext.ctypes.data, ctypes.byref(n_ext),
                                           pool.ctypes.data, ctypes.byref(n_pool)))
    return op, ext, pool


def rteaal_design_specialized_source(netlist: bytes, fuse_mux_chains: bool = False) -> str:
    """The design-specialised kernel's generated CUDA source (host only)."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    n = ctypes.c_size_t()
    _check(lib().rteaal_design_specialized_source(netlist, len(netlist), ctypes.byref(opts), None, 0,
                                                  ctypes.byref(n)))
    out = ctypes.create_string_buffer(max(n.value, 1))
    _check(lib().rteaal_design_specialized_source(netlist, len(netlist), ctypes.byref(opts), out, n.value,
                                                  ctypes.byref(n)))
    return out.raw[:n.value].decode()


def rteaal_design_specialize_host(netlist: bytes, fuse_mux_chains: bool = False) -> dict:
    """Generate and compile the design-specialised kernel on the host (no device):
    the compiled image's size and the generation + compile time."""
    opts = rteaal_load_opts()
    opts.device = -1
    opts.fuse_mux_chains = int(bool(fuse_mux_chains))
    nbytes, us = _U64(), _U64()
    _check(lib().rteaal_design_specialize_host(netlist, len(netlist), ctypes.byref(opts), ctypes.byref(nbytes),
                                               ctypes.byref(us)))
    return {"cubin_bytes": nbytes.value, "compile_us": us.value}


def rteaal_design_signals(design: int, n_signals: int) -> np.ndarray:
    """bool [n_signals]: True where the signal holds a row (False: fused away)."""
    out = np.zeros(n_signals, np.uint8)
    _check(lib().rteaal_design_signals(design, out.ctypes.data, n_signals))
    return out.astype(bool)


def rteaal_design_free(design: int):
    _check(lib().rteaal_design_free(design))


def rteaal_sim_create(design: int, n_instances: int, opts: rteaal_sim_opts | None = None) -> int:
    out = _P()
    _check(lib().rteaal_sim_create(design, n_instances,
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(out)))
    return out.value


def rteaal_sim_info(sim: int) -> dict:
    st = rteaal_sim_stats()
    _check(lib().rteaal_sim_info(sim, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in st._fields_}


def rteaal_sim_destroy(sim: int):
    lib().rteaal_sim_destroy(sim)


def rteaal_sim_configure(sim: int, opts: rteaal_sim_opts):
    _check(lib().rteaal_sim_configure(sim, ctypes.byref(opts)))


def rteaal_sim_autotune(sim: int, cycles_per_trial: int = 1, kernel_mask: int = 0,
                        max_trials: int = 256, stream=None) -> list[dict]:
    buf = (rteaal_tune_trial * max_trials)()
    n = _U32(0)
    _check(lib().rteaal_sim_autotune(sim, cycles_per_trial, kernel_mask, buf, max_trials,
                                     ctypes.byref(n), _stream_ptr(stream)))
    return [{f: getattr(buf[i], f) for f, _ in rteaal_tune_trial._fields_}
            for i in range(min(n.value, max_trials))]


def rteaal_sim_footprint(design: int, n_instances: int) -> int:
    return int(lib().rteaal_sim_footprint(design, n_instances))


def rteaal_step(sim: int, cycles: rteaal_cycles, stimulus: rteaal_stimulus,
                probes: rteaal_probes | None, flags: int, stream) -> None:
    _check(lib().rteaal_step(sim, ctypes.byref(cycles), ctypes.byref(stimulus),
                             ctypes.byref(probes) if probes is not None else None, flags,
                             _stream_ptr(stream)))


def rteaal_sim_reset_lanes(sim: int, inst_begin: int, n_inst: int, xorshift_seed=None, stream=None):
    seed = None
    if xorshift_seed is not None:
        seed = np.ascontiguousarray(xorshift_seed, np.uint64)
    _check(lib().rteaal_sim_reset_lanes(sim, inst_begin, n_inst,
                                        None if seed is None else seed.ctypes.data, _stream_ptr(stream)))


def rteaal_sim_activity(sim: int, stream=None) -> tuple[int, int]:
    ev, sk = _U64(0), _U64(0)
    _check(lib().rteaal_sim_activity(sim, ctypes.byref(ev), ctypes.byref(sk), _stream_ptr(stream)))
    return int(ev.value), int(sk.value)


def rteaal_sync(sim: int, stream=None):
    _check(lib().rteaal_sync(sim, _stream_ptr(stream)))


def rteaal_state_read(sim: int, signals, inst_begin: int, n_inst: int, stream=None) -> np.ndarray:
    sig = np.ascontiguousarray(np.asarray(signals, np.uint32).reshape(-1))
    out = np.zeros((sig.size, n_inst), np.uint64)
    _check(lib().rteaal_state_read(sim, _np_ptr(sig, _U32), sig.size, inst_begin, n_inst,
                                   out.ctypes.data, _stream_ptr(stream)))
    return out


def rteaal_state_write(sim: int, signals, inst_begin: int, values: np.ndarray, stream=None):
    sig = np.ascontiguousarray(np.asarray(signals, np.uint32).reshape(-1))
    v = np.ascontiguousarray(values, np.uint64)
    if v.ndim != 2 or v.shape[0] != sig.size:
        raise ValueError("values must be [n_signals][n_instances]")
    _check(lib().rteaal_state_write(sim, _np_ptr(sig, _U32), sig.size, inst_begin, v.shape[1],
                                    v.ctypes.data, _stream_ptr(stream)))


def rteaal_mem_read(sim: int, inst_begin: int, n_inst: int, words: int, stream=None) -> np.ndarray:
    out = np.zeros((words, n_inst), np.uint64)
    _check(lib().rteaal_mem_read(sim, inst_begin, n_inst, out.ctypes.data, _stream_ptr(stream)))
    return out


def rteaal_mem_write(sim: int, inst_begin: int, values: np.ndarray, stream=None):
    v = np.ascontiguousarray(values, np.uint64)
    _check(lib().rteaal_mem_write(sim, inst_begin, v.shape[1], v.ctypes.data, _stream_ptr(stream)))


def rteaal_stim_state_read(sim: int, inst_begin: int, n_inst: int, n_inputs: int,
                           stream=None) -> np.ndarray:
    out = np.zeros((n_inputs, n_inst), np.uint64)
    _check(lib().rteaal_stim_state_read(sim, inst_begin, n_inst, out.ctypes.data,
                                        _stream_ptr(stream)))
    return out


def rteaal_stim_state_write(sim: int, inst_begin: int, values: np.ndarray, stream=None):
    v = np.ascontiguousarray(values, np.uint64)
    _check(lib().rteaal_stim_state_write(sim, inst_begin, v.shape[1], v.ctypes.data,
                                         _stream_ptr(stream)))


def rteaal_step_static(design: int, state, mem, xs, n_lanes: int, cycles=None,
                       uniform_cycles: int = 0, stim_mode: int = RTEAAL_STIM_XORSHIFT,
                       flags: int = 0, stream=None):
    """Allocation-free step over caller-owned device buffers (see include/rteaal.h)."""
    keep = None
    cptr = None
    if cycles is not None:
        keep = np.ascontiguousarray(cycles, np.uint32)
        cptr = _np_ptr(keep, _U32)
    _check(lib().rteaal_step_static(design, _dev_ptr(state), _dev_ptr(mem), _dev_ptr(xs), n_lanes,
                                    cptr, uniform_cycles, stim_mode, flags, _stream_ptr(stream)))
    del keep


def rteaal_last_error() -> str:
    return lib().rteaal_last_error().decode(errors="replace")


# ------------------------------------------------------------ convenience objects
class Design:
    """A loaded netlist (owns the handle)."""

    def __init__(self, netlist: bytes, use_torch_allocator: bool = True, device: int = -1,
                 fuse_mux_chains: bool = False):
        self._opts = rteaal_load_opts()
        self._opts.device = device
        self._opts.fuse_mux_chains = int(fuse_mux_chains)
        if use_torch_allocator:
            self._alloc = torch_allocator()
            self._opts.allocator = ctypes.pointer(self._alloc)
        self.handle = rteaal_design_load(netlist, self._opts)
        self.info = rteaal_design_info(self.handle)

    def footprint(self, n_instances: int) -> int:
        return rteaal_sim_footprint(self.handle, n_instances)

    def specialize(self) -> float:
        """Compile the design-specialised kernel now; returns its generation + compile seconds."""
        us = _U64(0)
        _check(lib().rteaal_design_specialize(self.handle, ctypes.byref(us)))
        return us.value / 1e6

    def present_signals(self) -> np.ndarray:
        """Ids of the signals that hold a row (all of them unless fusion absorbed some)."""
        return np.flatnonzero(rteaal_design_signals(self.handle, self.info["n_signals"])).astype(np.uint32)

    def close(self):
        if self.handle:
            rteaal_design_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """n_instances independent instances of a design, resident on the device.

    kernel: "grid" (persistent, the whole GPU walks each layer: the batched form),
    "tile", "stream", "layer" / "layer_graph" (the plain form), "cluster", "flow"
    (one instance or a few: no barrier between layers; tile_lanes = items per warp),
    "specialized" or "auto"; the state is the same in every form, so configure()
    may switch between steps."""

    def __init__(self, design: Design, n_instances: int, kernel: str | int = "auto",
                 xorshift_seed: np.ndarray | None = None, expected_cycles=None,
                 tile_lanes: int = 0, threads: int = 0, ctas_per_sm: int = 0, unroll: int = 0,
                 lanes_per_thread: int = 0, use_torch_allocator: bool = True, activity: bool = False,
                 cluster_ctas: int = 0, cluster_resident: int = 0):
        self.design = design
        self.n = n_instances
        o = rteaal_sim_opts()
        o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        o.tile_lanes, o.threads, o.ctas_per_sm, o.unroll = tile_lanes, threads, ctas_per_sm, unroll
        o.lanes_per_thread = lanes_per_thread
        o.activity = int(activity)
        o.cluster_ctas = cluster_ctas
        o.cluster_resident = cluster_resident
        keep: list[Any] = []
        if use_torch_allocator:
            self._alloc = torch_allocator()
            o.allocator = ctypes.pointer(self._alloc)
        if xorshift_seed is not None:
            xs = np.ascontiguousarray(xorshift_seed, np.uint64)
            if xs.shape != (design.info["n_inputs"], n_instances):
                raise ValueError("xorshift_seed must be [n_inputs][n_instances]")
            keep.append(xs)
            o.xorshift_seed = _np_ptr(xs, _U64)
        if expected_cycles is not None:
            ec = np.ascontiguousarray(expected_cycles, np.uint32)
            if ec.size != n_instances:
                raise ValueError("expected_cycles must have one entry per instance")
            keep.append(ec)
            o.expected_cycles = _np_ptr(ec, _U32)
        self.handle = rteaal_sim_create(design.handle, n_instances, o)

    @property
    def info(self) -> dict:
        """Instance / lane counts, launch configuration and the last step's span (live)."""
        return rteaal_sim_info(self.handle)

    def step(self, cycles, stimulus: str = "hold", values=None, reset: bool = False,
             probes=None, probe_mode: str = "last", probe_out=None, stream=None,
             reset_per_instance=None, change_capacity: int = 1 << 16):
        """cycles: int or per-instance uint32 array.  values: BUFFER stimulus
        [cycles][n_inputs][n] as a device tensor / pointer, or a numpy array (host).
        probes: signal ids; probe_out: device tensor or None (returns a numpy array)."""
        cyc = rteaal_cycles()
        keep = []
        if np.isscalar(cycles):
            cyc.uniform = int(cycles)
        else:
            pc = np.ascontiguousarray(cycles, np.uint32)
            if pc.size != self.n:
                raise ValueError("per-instance cycles must have one entry per instance")
            keep.append(pc)
            cyc.per_instance = _np_ptr(pc, _U32)
        if reset_per_instance is not None:
            rp = np.ascontiguousarray(reset_per_instance, np.uint32)
            if rp.size != self.n:
                raise ValueError("reset_per_instance must have one entry per instance")
            keep.append(rp)
            cyc.reset_per_instance = _np_ptr(rp, _U32)
        st = rteaal_stimulus()
        st.mode = {"hold": 0, "xorshift": 1, "buffer": 2}[stimulus]
        if values is not None:
            if isinstance(values, np.ndarray):
                v = np.ascontiguousarray(values, np.uint64)
                ncyc = int(np.max(cycles)) if not np.isscalar(cycles) else int(cycles)
                if v.size < ncyc * int(self.design.info["n_inputs"]) * self.n:
                    raise ValueError("stimulus values must be [cycles][n_inputs][n_instances]")
                keep.append(v)
                st.values, st.values_on_host = int(v.ctypes.data), 1
            else:
                st.values, st.values_on_host = _dev_ptr(values), 0
        pr = None
        host_out = None
        if probes is not None and len(probes):
            sig = np.ascontiguousarray(np.asarray(probes, np.uint32))
            keep.append(sig)
            pr = rteaal_probes()
            pr.signals, pr.n = _np_ptr(sig, _U32), sig.size
            pr.mode = {"last": 0, "every": 1, "changes": 2}[probe_mode]
            if probe_mode == "changes":
                recs = np.zeros(change_capacity, CHANGE_DTYPE)
                count = np.zeros(1, np.uint64)
                pr.out, pr.out_on_host = int(recs.ctypes.data), 1
                pr.capacity = change_capacity
                pr.count = _np_ptr(count, _U64)
                rteaal_step(self.handle, cyc, st, pr, RTEAAL_STEP_RESET if reset else 0, stream)
                n = int(count[0])
                return recs[:min(n, change_capacity)], n
            if probe_out is None:
                ncyc = int(np.max(cycles)) if not np.isscalar(cycles) else int(cycles)
                rows = ncyc if probe_mode == "every" else 1
                host_out = np.zeros((rows, sig.size, self.n), np.uint64)
                pr.out, pr.out_on_host = int(host_out.ctypes.data), 1
            else:
                pr.out, pr.out_on_host = _dev_ptr(probe_out), 0
        rteaal_step(self.handle, cyc, st, pr, RTEAAL_STEP_RESET if reset else 0, stream)
        if host_out is not None:
            return host_out if probe_mode == "every" else host_out[0]
        return None

    def sync(self, stream=None):
        rteaal_sync(self.handle, stream)

    def activity(self, stream=None) -> tuple[int, int]:
        """(items evaluated, items skipped) since creation (activity-aware sims)."""
        return rteaal_sim_activity(self.handle, stream)

    def configure(self, kernel: str | int = "auto", tile_lanes: int = 0, threads: int = 0,
                  ctas_per_sm: int = 0, unroll: int = 0, lanes_per_thread: int = 0, cluster_ctas: int = 0,
                  cluster_resident: int = 0):
        o = rteaal_sim_opts()
        o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        o.tile_lanes, o.threads, o.ctas_per_sm, o.unroll = tile_lanes, threads, ctas_per_sm, unroll
        o.lanes_per_thread = lanes_per_thread
        o.cluster_ctas = cluster_ctas
        o.cluster_resident = cluster_resident
        rteaal_sim_configure(self.handle, o)

    def autotune(self, cycles_per_trial: int = 1, kernels=None, stream=None) -> list[dict]:
        """Time candidate launch configurations; keep the fastest; state is restored."""
        mask = 0
        for k in kernels or []:
            mask |= 1 << (KERNELS[k] if isinstance(k, str) else int(k))
        return rteaal_sim_autotune(self.handle, cycles_per_trial, mask, stream=stream)

    def read(self, signals=None, inst_begin: int = 0, n_inst: int | None = None, stream=None):
        if signals is None:
            signals = np.arange(self.design.info["n_signals"], dtype=np.uint32)
        return rteaal_state_read(self.handle, signals, inst_begin,
                                 self.n - inst_begin if n_inst is None else n_inst, stream)

    def write(self, signals, values: np.ndarray, inst_begin: int = 0, stream=None):
        rteaal_state_write(self.handle, signals, inst_begin, values, stream)

    def read_mem(self, inst_begin: int = 0, n_inst: int | None = None, stream=None):
        return rteaal_mem_read(self.handle, inst_begin, self.n - inst_begin if n_inst is None else n_inst,
                               int(self.design.info["mem_words_total"]), stream)

    def write_mem(self, values: np.ndarray, inst_begin: int = 0, stream=None):
        if np.ndim(values) != 2 or np.shape(values)[0] != int(self.design.info["mem_words_total"]):
            raise ValueError("memory words must be [mem_words_total][n_instances]")
        rteaal_mem_write(self.handle, inst_begin, values, stream)

    def reset_lanes(self, inst_begin: int, n_inst: int, xorshift_seed=None, stream=None):
        if xorshift_seed is not None and np.shape(xorshift_seed) != (int(self.design.info["n_inputs"]), n_inst):
            raise ValueError("xorshift_seed must be [n_inputs][n_inst]")
        rteaal_sim_reset_lanes(self.handle, inst_begin, n_inst, xorshift_seed, stream)

    def read_stim_state(self, inst_begin: int = 0, n_inst: int | None = None, stream=None):
        return rteaal_stim_state_read(self.handle, inst_begin,
                                      self.n - inst_begin if n_inst is None else n_inst,
                                      int(self.design.info["n_inputs"]), stream)

    def write_stim_state(self, values: np.ndarray, inst_begin: int = 0, stream=None):
        if np.ndim(values) != 2 or np.shape(values)[0] != int(self.design.info["n_inputs"]):
            raise ValueError("xorshift states must be [n_inputs][n_instances]")
        rteaal_stim_state_write(self.handle, inst_begin, values, stream)

    def close(self):
        if self.handle:
            rteaal_sim_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/rteaal.h declares, and rejects malformed netlists
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    rtbuild.build()
    return rt.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "rteaal.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rteaal_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(L):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(rt.EXPORTS)


def test_malformed_netlists_rejected_on_host(L):
    good = synth.generate(synth.DesignSpec(n_ops=50, n_regs=4, depth=4, seed=1)).to_bytes()
    out = ctypes.c_void_p()
    for bad in [good[:-1], b"XXXX" + good[4:], good[:20]]:
        rc = L.rteaal_design_load(bad, len(bad), None, ctypes.byref(out))
        assert rc == rt.RTEAAL_E_FORMAT
        assert out.value is None
    nl = synth.Netlist.from_bytes(good)
    nl.args[3] = nl.n_signals + 1
    b = nl.to_bytes()
    assert L.rteaal_design_load(b, len(b), None, ctypes.byref(out)) == rt.RTEAAL_E_FORMAT
    assert b"topological" in L.rteaal_last_error()
    nl = synth.Netlist.from_bytes(good)
    nl.op_width[0] = 65
    b = nl.to_bytes()
    assert L.rteaal_design_load(b, len(b), None, ctypes.byref(out)) == rt.RTEAAL_E_FORMAT


def test_null_arguments(L):
    out = ctypes.c_void_p()
    assert L.rteaal_design_load(None, 0, None, ctypes.byref(out)) == rt.RTEAAL_E_INVALID
    assert L.rteaal_design_free(None) == rt.RTEAAL_OK
    assert L.rteaal_sim_footprint(None, 5) == 0


def test_fast_division_formula():
    """The multiply-high division the kernels use to split item indices."""
    rng = np.random.default_rng(0)
    ns = np.concatenate([np.arange(5000), rng.integers(0, 2**31, 20000), [2**31 - 1, 2**32 - 1]])
    for d in list(range(1, 300)) + [1000, 4096, 6553, 65536, 99991, 2**20 + 7]:
        l = (d - 1).bit_length()
        m = ((1 << 32) * ((1 << l) - d)) // d + 1
        assert m < 2**32
        q = ((((ns.astype(object) * m) >> 32) + ns.astype(object)) >> l)
        assert (q == ns.astype(object) // d).all(), d

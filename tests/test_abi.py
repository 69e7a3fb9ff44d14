"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/rteaal.h declares, rejects malformed netlists before
touching the device, and a plain C program can include the header and link."""
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


def test_header_is_plain_c_and_links(L, tmp_path):
    """A C11 program includes the header (no C++ constructs, no warnings under
    -pedantic), links against the library and calls a host-only entry point."""
    import subprocess
    src = tmp_path / "consumer.c"
    src.write_text(
        '#include "rteaal.h"\n'
        '#include <stdio.h>\n'
        'int main(void) {\n'
        '  rteaal_design_stats st;\n'
        '  const char bad[4] = {0, 0, 0, 0};\n'
        '  int rc = rteaal_design_lower(bad, sizeof bad, NULL, &st, NULL, 0);\n'
        '  printf("%d %s\\n", rc, rteaal_last_error());\n'
        '  return rc == RTEAAL_E_FORMAT ? 0 : 1;\n'
        '}\n')
    libdir = os.path.dirname(rt.LIB_PATH)
    exe = tmp_path / "consumer"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-o", str(exe), str(src), "-L", libdir, "-lrteaal",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("%d " % rt.RTEAAL_E_FORMAT)

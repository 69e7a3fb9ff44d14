"""The design-specialised kernel's generator on the host (no GPU): the
straight-line CUDA it writes for a netlist compiles for sm_103a with NVRTC for
every feature it has to express -- memories and write ports, fused mux chains,
clock domains, registers fed straight from inputs and constants, a design
without ops -- and designs beyond its size limit are refused.  Whether the
compiled kernel computes the right values is the GPU parity tests' job."""
import pytest

import paper_2601_18140_gb300 as rt
import synth
from paper_2601_18140_gb300 import build as rtbuild
from synth import Builder, DesignSpec


@pytest.fixture(scope="module", autouse=True)
def _lib():
    rtbuild.build()


def compiles(nl: synth.Netlist, fuse: bool = False) -> dict:
    r = rt.rteaal_design_specialize_host(nl.to_bytes(), fuse_mux_chains=fuse)
    assert r["cubin_bytes"] > 0
    return r


def test_random_design_with_memories():
    compiles(synth.generate(DesignSpec(n_ops=300, n_regs=20, depth=6, seed=3, n_mems=2, mem_words=8,
                                       mem_write_ports=2)))


@pytest.mark.parametrize("fuse", [False, True])
def test_mux_chains(fuse):
    nl = synth.generate(DesignSpec(n_ops=300, n_regs=20, depth=6, n_inputs=4, seed=71,
                                   input_widths=(8, 32, 1, 64), mux_chain_frac=0.7))
    if fuse:
        assert rt.rteaal_design_lower(nl.to_bytes(), fuse_mux_chains=True)[0]["n_fused"] > 0
    compiles(nl, fuse)


def test_clock_domains_and_degenerate_designs():
    b = Builder()
    i0 = b.input(8)
    k = b.const(16, 0xBEEF)
    r0, r1, r2 = b.reg(8), b.reg(16), b.reg(8)
    b.connect(r0, b.op("ADD", 8, r0, i0))
    b.connect(r1, k)
    b.connect(r2, i0)
    b.clock(r0, b.domain(4, 1))
    b.clock(r2, b.domain(2, 0))
    compiles(b.build())
    b = Builder()
    b.input(1)
    compiles(b.build())


def test_size_limit_and_malformed_input():
    nl = synth.generate(DesignSpec(n_ops=16_385, n_regs=16, depth=4, seed=1))
    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_design_specialize_host(nl.to_bytes())
    assert ei.value.code == rt.RTEAAL_E_UNSUPPORTED
    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_design_specialize_host(nl.to_bytes()[:-3])
    assert ei.value.code == rt.RTEAAL_E_FORMAT

"""The allocation-free entry point, rteaal_step_static.

Callers that cannot allocate device memory themselves (their device memory
is owned by another allocator, or libraries may not call cudaMalloc) run the
grid form over buffers they own; the entry point's only scratch is a
file-scope device array.  This test checks, through the C ABI, that two calls
in a row give exactly the state of the regular entry point (rteaal_step) on
the same inputs: integer simulation, so the tolerance is bit-exactness.
Collected last on purpose (file name), and independent of the other tests.
"""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt
import synth
from synth import DesignSpec

pytestmark = pytest.mark.gpu


def slot_of_signal(nl: synth.Netlist) -> np.ndarray:
    """Row of every signal in the state layout: pool rows are the signal ids; op
    rows follow level, then (opcode, width), then netlist order."""
    n = nl.n_signals
    lvl = np.zeros(n, np.int64)
    for k in range(nl.n_ops):
        a = nl.op_args(k)
        lvl[nl.op_base + k] = 1 + (lvl[a].max() if a.size else 0)
    key = np.lexsort((np.arange(nl.n_ops), nl.op_width, nl.op_code, lvl[nl.op_base:]))
    slot = np.arange(n, dtype=np.int64)
    slot[nl.op_base + key] = nl.op_base + np.arange(nl.n_ops)
    return slot


def compact_rows(nl: synth.Netlist):
    """Width class and per-lane byte offset of every slot (the compact layout of
    include/rteaal.h: class-3 rows first, then 2, 1, 0; pool rows before op rows)."""
    slot = slot_of_signal(nl)
    width = np.zeros(nl.n_signals, np.int64)
    width[slot] = nl.signal_widths()
    cls = np.select([width <= 8, width <= 16, width <= 32], [0, 1, 2], 3)
    cnt = [int((cls == k).sum()) for k in range(4)]
    nxt = {3: 0, 2: 8 * cnt[3]}
    nxt[1] = nxt[2] + 4 * cnt[2]
    nxt[0] = nxt[1] + 2 * cnt[1]
    lane_bytes = nxt[0] + cnt[0]
    off = np.zeros(nl.n_signals, np.int64)
    for sl in range(nl.n_signals):
        k = int(cls[sl])
        off[sl] = nxt[k]
        nxt[k] += 1 << k
    return slot, cls, off, lane_bytes


def decode(buf: np.ndarray, cls, off, n: int) -> np.ndarray:
    """Rows of a compact state buffer (uint8) as uint64 [n_slots][n]."""
    out = np.zeros((cls.size, n), np.uint64)
    dt = {0: np.uint8, 1: np.uint16, 2: np.uint32, 3: np.uint64}
    for sl in range(cls.size):
        k = int(cls[sl])
        start = int(off[sl]) * n
        out[sl] = buf[start:start + (n << k)].view(dt[k]).astype(np.uint64)
    return out


def test_static_step_matches_regular_step():
    import torch

    nl = synth.generate(DesignSpec(n_ops=1500, n_regs=80, depth=12, n_inputs=4,
                                   input_widths=(8, 32, 64, 1), seed=77, n_mems=3, mem_words=16))
    # every register D and write-port signal is an op output: no inserted copy rows
    assert (nl.reg_d >= nl.op_base).all() and (nl.wport[:, 1:] >= nl.op_base).all()
    n = 256
    xs = synth.xorshift_seeds(77, nl.n_inputs, n)
    d = rt.Design(nl.to_bytes())
    info = d.info
    assert info["n_slots"] == nl.n_signals

    # regular path
    sim = rt.Sim(d, n, kernel="grid", xorshift_seed=xs)
    assert sim.info["n_lanes"] == n

    # caller-owned buffers in the documented layout
    slot, cls, off, lane_bytes = compact_rows(nl)
    assert lane_bytes == info["state_bytes_per_lane"]
    dev = torch.device("cuda")
    img = np.zeros(lane_bytes * n, np.uint8)
    dt = {0: np.uint8, 1: np.uint16, 2: np.uint32, 3: np.uint64}
    for c in range(nl.n_consts):
        sl = nl.const_base + c
        k = int(cls[sl])
        start = int(off[sl]) * n
        img[start:start + (n << k)] = np.full(n, nl.const_value[c], dt[k]).view(np.uint8)
    state = torch.from_numpy(img).to(dev)
    mem = torch.zeros((int(info["mem_words_total"]), n), dtype=torch.int64, device=dev)
    xsd = torch.from_numpy(xs.copy().view(np.int64)).to(dev)
    torch.cuda.synchronize()

    slot = slot_of_signal(nl)
    budgets = (5 + (np.arange(n) * 7) % 23).astype(np.uint32)

    # call 1: the reset cycle; call 2: uneven cycle counts per instance
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, None, 1, rt.RTEAAL_STIM_XORSHIFT,
                          rt.RTEAAL_STEP_RESET)
    sim.step(1, stimulus="xorshift", reset=True)
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, budgets, 0, rt.RTEAAL_STIM_XORSHIFT, 0)
    sim.step(budgets, stimulus="xorshift")

    got = decode(state.cpu().numpy(), cls, off, n)[slot]
    exp = sim.read()
    assert np.array_equal(got, exp)
    assert np.array_equal(mem.cpu().numpy().view(np.uint64), sim.read_mem())
    assert np.array_equal(xsd.cpu().numpy().view(np.uint64), sim.read_stim_state())

    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_step_static(d.handle, state, mem, xsd, rt.STATIC_MAX_LANES + 1, None, 1)
    assert ei.value.code == rt.RTEAAL_E_INVALID
    sim.close()
    d.close()

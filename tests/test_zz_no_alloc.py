"""The allocation-free entry point, rteaal_step_static.

Some callers cannot allocate device memory at all: their device memory belongs
to another allocator or framework that forbids libraries to call cudaMalloc /
cudaFree (or has already handed out every byte).  They run the grid form over
buffers they own; the entry point's only scratch is a file-scope device array.
This test builds those buffers from the layout the header documents (not from
the library), runs two calls in a row through the C ABI -- a reset cycle, then
uneven per-instance cycle counts -- and checks the state, memories and
stimulus states against the regular entry point (rteaal_step) and against the
oracle: integer simulation, so the tolerance is bit-exactness.  It covers the
two-lanes-per-thread path (even lane count, 16-byte aligned buffers) and the
one-lane path (odd count), xorshift and held inputs, ops with more than three
operands (side-array operand lists) among narrow and wide ones, the size
limit, and a bounded barrier wait that gives up.  Collected last on purpose
(file name), and independent of the other tests.
"""
import numpy as np
import pytest

import oracle
import paper_2601_18140_gb300 as rt
import synth
from synth import OP, DesignSpec, Netlist

pytestmark = pytest.mark.gpu


def with_wide_folds(nl: Netlist, seed: int) -> Netlist:
    """The generated design plus variadic ops with four to seven operands (AND /
    XOR / ADD folds, MUXCHAIN), narrow and wide, that some registers load."""
    rng = np.random.default_rng(seed)
    w = nl.signal_widths().astype(np.int64)
    n_sig = nl.n_signals
    narrow_pool = np.flatnonzero(w <= 32)
    any_pool = np.arange(n_sig)
    codes, widths, args = [], [], []
    for k in range(48):
        narrow = k % 2 == 0
        pool = narrow_pool if narrow else any_pool
        kind = k % 4
        if kind == 3:                                  # MUXCHAIN s0, v0, s1, v1, [s2, v2,] default
            n = 5 if k % 8 == 3 else 7
            code = OP["MUXCHAIN"]
        else:
            n = 4 + k % 4
            code = [OP["AND"], OP["XOR"], OP["ADD"]][kind]
        codes.append(code)
        widths.append(int(rng.choice([8, 16, 32])) if narrow else int(rng.choice([33, 48, 64])))
        args.append(rng.choice(pool, n).astype(np.uint32))
    op_code = np.concatenate([nl.op_code, np.array(codes, np.uint8)])
    op_width = np.concatenate([nl.op_width, np.array(widths, np.uint8)])
    z = np.zeros(len(codes), np.uint8)
    argoff = list(nl.op_argoff)
    for a in args:
        argoff.append(argoff[-1] + len(a))
    new_ops = nl.op_base + nl.n_ops + np.arange(len(codes))
    reg_d = nl.reg_d.copy()
    reg_d[:len(codes)] = new_ops[:min(len(codes), nl.n_regs)]     # registers load the new ops
    return Netlist(nl.input_width, nl.reg_width, reg_d, nl.reg_init, nl.const_width, nl.const_value,
                   op_code, op_width, np.concatenate([nl.op_p0, z]), np.concatenate([nl.op_p1, z]),
                   np.array(argoff, np.uint32), np.concatenate([nl.args] + args).astype(np.uint32),
                   nl.mem_words, nl.mem_width, nl.wport, nl.dom_period, nl.dom_phase, nl.reg_domain)


def slot_of_signal(nl: Netlist) -> np.ndarray:
    """Row of every signal in the documented layout: pool rows are the signal
    ids; op rows by level, then ops with at most three operands before the
    others, among those narrow before wide, then (opcode, width), then netlist
    order."""
    w = nl.signal_widths().astype(np.int64)
    lvl = np.zeros(nl.n_signals, np.int64)
    ext = np.zeros(nl.n_ops, np.int64)
    wide = np.zeros(nl.n_ops, np.int64)
    for k in range(nl.n_ops):
        a = nl.op_args(k).astype(np.int64)
        lvl[nl.op_base + k] = 1 + (lvl[a].max() if a.size else 0)
        ext[k] = a.size > 3
        c, p0 = int(nl.op_code[k]), int(nl.op_p0[k])
        wide[k] = (not ext[k]) and (nl.op_width[k] > 32 or c == OP["MEMRD"] or (c == OP["BITS"] and p0 >= 32)
                                    or (c == OP["ANDR"] and p0 > 32) or bool((w[a] > 32).any()))
    key = np.lexsort((np.arange(nl.n_ops), nl.op_width, nl.op_code, wide, ext, lvl[nl.op_base:]))
    slot = np.arange(nl.n_signals, dtype=np.int64)
    slot[nl.op_base + key] = nl.op_base + np.arange(nl.n_ops)
    return slot


def compact_rows(nl: Netlist):
    """Width class and per-lane byte offset of every slot (the compact layout:
    class-3 rows first, then 2, 1, 0; inside a class, slot order)."""
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


DT = {0: np.uint8, 1: np.uint16, 2: np.uint32, 3: np.uint64}


def decode(buf: np.ndarray, cls, off, n: int) -> np.ndarray:
    """Rows of a compact state buffer (uint8) as uint64 [n_slots][n]."""
    out = np.zeros((cls.size, n), np.uint64)
    for sl in range(cls.size):
        k = int(cls[sl])
        start = int(off[sl]) * n
        out[sl] = buf[start:start + (n << k)].view(DT[k]).astype(np.uint64)
    return out


def design() -> Netlist:
    nl = synth.generate(DesignSpec(n_ops=1500, n_regs=80, depth=12, n_inputs=4,
                                   input_widths=(8, 32, 64, 1), seed=77, n_mems=3, mem_words=16))
    return with_wide_folds(nl, 77)


@pytest.mark.parametrize("n,stim", [(256, "xorshift"), (255, "xorshift"), (255, "hold"), (256, "hold")])
def test_static_step_matches_regular_step_and_oracle(n, stim):
    import torch

    nl = design()
    # every register D and write-port signal is an op output: no inserted copy rows
    assert (nl.reg_d >= nl.op_base).all() and (nl.wport[:, 1:] >= nl.op_base).all()
    assert max(len(nl.op_args(k)) for k in range(nl.n_ops)) > 3
    mode = {"xorshift": rt.RTEAAL_STIM_XORSHIFT, "hold": rt.RTEAAL_STIM_HOLD}[stim]
    omode = {"xorshift": oracle.STIM_XORSHIFT, "hold": oracle.STIM_HOLD}[stim]
    xs = synth.xorshift_seeds(77, nl.n_inputs, n)
    d = rt.Design(nl.to_bytes())
    info = d.info
    assert info["n_slots"] == nl.n_signals

    # regular path (its own device allocations)
    sim = rt.Sim(d, n, kernel="grid", xorshift_seed=xs)

    # caller-owned buffers in the documented layout
    slot, cls, off, lane_bytes = compact_rows(nl)
    assert lane_bytes == info["state_bytes_per_lane"]
    dev = torch.device("cuda")
    img = np.zeros(lane_bytes * n, np.uint8)
    for c in range(nl.n_consts):
        sl = nl.const_base + c
        k = int(cls[sl])
        start = int(off[sl]) * n
        img[start:start + (n << k)] = np.full(n, nl.const_value[c], DT[k]).view(np.uint8)
    state = torch.from_numpy(img).to(dev)
    mem = torch.zeros((int(info["mem_words_total"]), n), dtype=torch.int64, device=dev)
    xsd = torch.from_numpy(xs.copy().view(np.int64)).to(dev)
    torch.cuda.synchronize()

    budgets = (5 + (np.arange(n) * 7) % 23).astype(np.uint32)
    orc = oracle.OracleSim(nl.to_bytes(), n)
    oxs = xs.copy()

    # call 1: the reset cycle (inputs driven by xorshift); call 2: uneven cycle
    # counts per instance, inputs held or driven as the case says
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, None, 1, rt.RTEAAL_STIM_XORSHIFT, rt.RTEAAL_STEP_RESET)
    sim.step(1, stimulus="xorshift", reset=True)
    orc.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=8)
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, budgets, 0, mode, 0)
    sim.step(budgets, stimulus=stim)
    orc.step(budgets, mode=omode, xs=oxs, threads=8)

    got = decode(state.cpu().numpy(), cls, off, n)[slot]
    assert np.array_equal(got, sim.read())
    assert np.array_equal(got, orc.read())
    gm = mem.cpu().numpy().view(np.uint64)
    assert np.array_equal(gm, sim.read_mem()) and np.array_equal(gm, orc.read_mem())
    gx = xsd.cpu().numpy().view(np.uint64)
    assert np.array_equal(gx, sim.read_stim_state()) and np.array_equal(gx, oxs)

    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_step_static(d.handle, state, mem, xsd, rt.STATIC_MAX_LANES + 1, None, 1)
    assert ei.value.code == rt.RTEAAL_E_INVALID
    sim.close()
    d.close()


def test_static_step_barrier_timeout_is_reported(monkeypatch):
    """A grid barrier wait that gives up (one arrival withheld, 0.2 s bound)
    returns RTEAAL_E_TIMEOUT; the next call, without the hook, runs normally."""
    import torch

    nl = design()
    n = 128
    d = rt.Design(nl.to_bytes())
    slot, cls, off, lane_bytes = compact_rows(nl)
    img = np.zeros(lane_bytes * n, np.uint8)
    for c in range(nl.n_consts):
        sl = nl.const_base + c
        k = int(cls[sl])
        img[int(off[sl]) * n:int(off[sl]) * n + (n << k)] = np.full(n, nl.const_value[c], DT[k]).view(np.uint8)
    state = torch.from_numpy(img).cuda()
    mem = torch.zeros((int(d.info["mem_words_total"]), n), dtype=torch.int64, device="cuda")
    xs = synth.xorshift_seeds(5, nl.n_inputs, n)
    xsd = torch.from_numpy(xs.copy().view(np.int64)).cuda()
    monkeypatch.setenv("RTEAAL_BARRIER_TIMEOUT_NS", "200000000")
    monkeypatch.setenv("RTEAAL_TEST_WITHHOLD_ARRIVAL", "1")
    with pytest.raises(rt.RteaalError) as ei:
        rt.rteaal_step_static(d.handle, state, mem, xsd, n, None, 3, rt.RTEAAL_STIM_XORSHIFT, 0)
    assert ei.value.code == rt.RTEAAL_E_TIMEOUT
    monkeypatch.delenv("RTEAAL_TEST_WITHHOLD_ARRIVAL")
    monkeypatch.delenv("RTEAAL_BARRIER_TIMEOUT_NS")
    # the device still works: a reset and a few cycles from fresh buffers equal the oracle
    state.copy_(torch.from_numpy(img).cuda())
    mem.zero_()
    xsd.copy_(torch.from_numpy(xs.copy().view(np.int64)).cuda())
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, None, 1, rt.RTEAAL_STIM_XORSHIFT, rt.RTEAAL_STEP_RESET)
    rt.rteaal_step_static(d.handle, state, mem, xsd, n, None, 9, rt.RTEAAL_STIM_XORSHIFT, 0)
    orc = oracle.OracleSim(nl.to_bytes(), n)
    oxs = xs.copy()
    orc.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=8)
    orc.step(9, mode=oracle.STIM_XORSHIFT, xs=oxs, threads=8)
    assert np.array_equal(decode(state.cpu().numpy(), cls, off, n)[slot], orc.read())
    d.close()

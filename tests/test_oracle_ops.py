"""Pins for the oracle's per-operation semantics (CPU only).

oracle.c computes with 64-bit wraparound, masks and shift guards; the
reference here is Python's unbounded-integer arithmetic reduced modulo 2^w
(oracle/pyeval.py) plus a few hand-checked values.  Exhaustive over every
operand value at widths 1, 4 and 8; sampled with edge values at 16, 32, 64.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle.pyeval import op_value
from synth import OP

BINARY = ["AND", "OR", "XOR", "ADD", "SUB", "MUL", "DSHL", "DSHR", "EQ", "NEQ", "LT", "LEQ",
          "GT", "GEQ"]
UNARY = ["COPY", "NOT", "ORR", "XORR"]


def _check(code, w, rows, p0=0, p1=0):
    rows = np.asarray(rows, dtype=np.uint64)
    got = oracle.eval_batch(code, w, rows, p0, p1)
    for i in range(rows.shape[0]):
        xs = [int(x) for x in rows[i]]
        exp = op_value(code, w, p0, p1, xs)
        assert int(got[i]) == exp, (code, w, p0, p1, xs, int(got[i]), exp)


def _all(w, k):
    vals = range(1 << w)
    return np.array(list(itertools.product(vals, repeat=k)), dtype=np.uint64)


@pytest.mark.parametrize("w", [1, 4, 8])
@pytest.mark.parametrize("name", BINARY)
def test_binary_exhaustive(name, w):
    rows = _all(w, 2)
    for wo in sorted({1, w, 2 * w if 2 * w <= 64 else 64}):
        _check(OP[name], wo, rows)


@pytest.mark.parametrize("w", [1, 4, 8])
@pytest.mark.parametrize("name", UNARY)
def test_unary_exhaustive(name, w):
    rows = _all(w, 1)
    for wo in sorted({1, w, 64}):
        _check(OP[name], wo, rows)


@pytest.mark.parametrize("w", [1, 4, 8])
def test_param_ops_exhaustive(w):
    rows = _all(w, 1)
    for k in [0, 1, w - 1, w, 63, 64, 200]:
        _check(OP["SHL"], w, rows, p0=k)
        _check(OP["SHL"], 64, rows, p0=k)
        _check(OP["SHR"], w, rows, p0=k)
    for hi in range(w):
        for lo in range(hi + 1):
            _check(OP["BITS"], hi - lo + 1, rows, p0=hi, p1=lo)
    _check(OP["ANDR"], 1, rows, p0=w)
    rows2 = _all(w, 2)
    _check(OP["CAT"], 2 * w, rows2, p0=w)


@pytest.mark.parametrize("w", [1, 4])
def test_mux_exhaustive(w):
    rows = _all(w, 3)
    _check(OP["MUX"], w, rows)
    _check(OP["MUXCHAIN"], w, rows)
    rows5 = _all(2, 5) if w == 1 else _all(1, 5)
    _check(OP["MUXCHAIN"], 2, rows5)


@pytest.mark.parametrize("w", [16, 32, 64])
def test_wide_sampled(w):
    rng = np.random.default_rng(1234 + w)
    edge = [0, 1, 2, (1 << w) - 1, 1 << (w - 1), (1 << (w - 1)) - 1]
    rnd = [int(x) for x in rng.integers(0, 1 << min(w, 63), size=40, dtype=np.uint64)]
    if w == 64:
        rnd += [int(x) | (1 << 63) for x in rnd[:20]]
    vals = edge + rnd
    rows2 = np.array(list(itertools.product(vals, repeat=2)), dtype=np.uint64)
    for name in BINARY:
        _check(OP[name], w, rows2)
    rows1 = np.array([[v] for v in vals + [63, 64, 65, 127, 128]], dtype=np.uint64)
    for name in UNARY:
        _check(OP[name], w, rows1)
    _check(OP["ANDR"], 1, rows1, p0=w)
    for k in [0, 1, 13, 31, 63]:
        _check(OP["SHL"], w, rows1, p0=k)
        _check(OP["SHR"], w, rows1, p0=k)
    _check(OP["BITS"], 8, rows1, p0=min(w - 1, 20), p1=min(w - 1, 20) - 7)
    rows3 = np.array([[s, a, b] for s in (0, 1, 2, 3) for a in vals[:8] for b in vals[:8]],
                     dtype=np.uint64)
    _check(OP["MUX"], w, rows3)


def test_hand_values():
    """A few values worked out by hand from the definitions."""
    ev = oracle.eval_one
    assert ev(OP["SUB"], 8, [3, 5]) == 254                 # 3 - 5 mod 2^8
    assert ev(OP["SUB"], 64, [0, 1]) == 2**64 - 1
    assert ev(OP["ADD"], 8, [200, 100]) == 44              # 300 mod 256
    assert ev(OP["MUL"], 16, [0xFFFF, 0xFFFF]) == 1        # (2^16-1)^2 mod 2^16
    assert ev(OP["MUL"], 64, [0xFFFFFFFF, 0xFFFFFFFF]) == 0xFFFFFFFE00000001
    assert ev(OP["NOT"], 4, [0b1010]) == 0b0101
    assert ev(OP["NOT"], 8, [0b1010]) == 0b11110101
    assert ev(OP["DSHL"], 64, [1, 63]) == 1 << 63
    assert ev(OP["DSHL"], 64, [1, 64]) == 0                # amount >= 64 gives 0
    assert ev(OP["DSHR"], 64, [1 << 63, 64]) == 0
    assert ev(OP["SHL"], 8, [0x81], p0=1) == 0x02
    assert ev(OP["SHR"], 8, [0x81], p0=7) == 1
    assert ev(OP["BITS"], 4, [0xABCD], p0=11, p1=8) == 0xB
    assert ev(OP["CAT"], 16, [0xAB, 0xCD], p0=8) == 0xABCD  # o0 in the high bits
    assert ev(OP["CAT"], 64, [0x1, 0x2], p0=64) == 0x2      # a << 64 leaves nothing
    assert ev(OP["LT"], 1, [2**64 - 1, 0]) == 0             # unsigned compare
    assert ev(OP["GT"], 1, [2**64 - 1, 0]) == 1
    assert ev(OP["ANDR"], 1, [0xF], p0=4) == 1
    assert ev(OP["ANDR"], 1, [0xF], p0=5) == 0
    assert ev(OP["XORR"], 1, [0b1011]) == 1
    assert ev(OP["ORR"], 1, [0]) == 0
    # mux: O=0 is the selector, bit 0 set picks O=1, clear picks O=2 (App. A)
    assert ev(OP["MUX"], 8, [1, 7, 9]) == 7
    assert ev(OP["MUX"], 8, [0, 7, 9]) == 9
    assert ev(OP["MUX"], 8, [2, 7, 9]) == 9                 # only bit 0 of the selector counts
    # mux chain: the first set selector wins, else the default (last operand)
    assert ev(OP["MUXCHAIN"], 8, [0, 1, 1, 2, 1, 3, 4]) == 2
    assert ev(OP["MUXCHAIN"], 8, [0, 1, 0, 2, 0, 3, 4]) == 4
    # variadic reducible ops fold in O order
    assert ev(OP["ADD"], 8, [100, 100, 100]) == 44
    assert ev(OP["XOR"], 8, [1, 2, 4, 8]) == 15

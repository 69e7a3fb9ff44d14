"""The pins have teeth: plausible mistakes planted in a copy of oracle.c (a
swapped operand, an inverted select, a dropped mask, a wrong shift constant,
reversed write-port priority, registers committed in place, ops evaluated out
of topological order, ...) each make at least one pin fail.  The mistakes are
planted in a temporary copy on the CPU; oracle.c itself is never touched."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_bruteforce as bf
from tests import test_oracle_circuits as circ
from tests import test_oracle_ops as ops

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text in oracle.c, replacement)
MUTANTS = [
    ("SUB operands swapped",
     "case O_SUB: r = v[a[0]] - v[a[1]];", "case O_SUB: r = v[a[1]] - v[a[0]];"),
    ("MUX select inverted",
     "r = (v[a[0]] & 1u) ? v[a[1]] : v[a[2]];", "r = (v[a[0]] & 1u) ? v[a[2]] : v[a[1]];"),
    ("result mask one bit short",
     "return r & mask_w(n->width[k]);", "return r & mask_w(n->width[k] > 1 ? n->width[k] - 1 : 1);"),
    ("BITS mask one bit short",
     "mask_w(p0 - p1 + 1)", "mask_w(p0 - p1)"),
    ("DSHL without the >= 64 guard",
     "r = y >= 64 ? 0 : x << y;", "r = x << (y & 63);"),
    ("MUXCHAIN last set selector wins",
     "{ r = v[a[2 * i + 1]]; break; }", "{ r = v[a[2 * i + 1]]; }"),
    ("xorshift middle shift 9 instead of 7",
     "x ^= x >> 7;", "x ^= x >> 9;"),
    ("inputs not masked to their width",
     "v[q] = val & mask_w(n->in_w[q]);", "v[q] = val;"),
    ("ops evaluated in reverse order",
     "for (uint32_t k = 0; k < n->no; k++) v[n->op_base + k] = eval_op(n, k, v, mem);",
     "for (uint32_t k = n->no; k-- > 0;) v[n->op_base + k] = eval_op(n, k, v, mem);"),
    ("reset ignores init values",
     "next[r] = n->reg_init[r] & mask_w(n->reg_w[r]);", "next[r] = 0;"),
    ("registers committed in place (no pre-edge copy)",
     "next[r] = v[n->reg_d[r]] & mask_w(n->reg_w[r]);",
     "next[r] = v[n->reg_base + r] = v[n->reg_d[r]] & mask_w(n->reg_w[r]);"),
    ("earlier write port wins",
     "for (uint32_t p = 0; p < n->nw; p++) {\n        const uint32_t *w = n->wport + 4ull * p;\n        if (v[w[1]] & 1u)",
     "for (uint32_t p = n->nw; p-- > 0;) {\n        const uint32_t *w = n->wport + 4ull * p;\n        if (v[w[1]] & 1u)"),
    ("memory read address masked short",
     "r = mem[n->mem_off[m] + (v[a[0]] & (uint64_t)(n->mem_words[m] - 1))];",
     "r = mem[n->mem_off[m] + (v[a[0]] & (uint64_t)(n->mem_words[m] - 2))];"),
    ("clock-domain phase subtracted",
     "(uint32_t)(j->ticks[i] + n->dom_phase[n->reg_dom[r]])",
     "(uint32_t)(j->ticks[i] - n->dom_phase[n->reg_dom[r]])"),
    ("domain counter not cleared by reset",
     "j->ticks[i] = j->reset ? 0u : j->ticks[i] + 1u;", "j->ticks[i] = j->ticks[i] + 1u;"),
]

# fast pins, run against every mutant
PINS = [
    ("op hand values", ops.test_hand_values),
    ("SUB exhaustive", lambda: ops.test_binary_exhaustive("SUB", 4)),
    ("DSHL exhaustive", lambda: ops.test_binary_exhaustive("DSHL", 4)),
    ("ADD exhaustive", lambda: ops.test_binary_exhaustive("ADD", 4)),
    ("parameterised ops", lambda: ops.test_param_ops_exhaustive(4)),
    ("mux / muxchain", lambda: ops.test_mux_exhaustive(4)),
    ("counter closed form", lambda: circ.test_counter_closed_form(8, 1000)),
    ("LFSR golden values", circ.test_lfsr_golden_values),
    ("xorshift = T^c s0", circ.test_xorshift_stimulus_matches_matrix_power),
    ("shift-register delay", lambda: circ.test_shift_register_delay(2)),
    ("register file vs dict", circ.test_register_file_matches_dict_model),
    ("two write ports", circ.test_two_write_ports_higher_index_wins),
    ("reset", circ.test_reset_sets_init_and_counts_as_a_cycle),
    ("clock domains", circ.test_clock_domains_count_their_ticks),
    ("brute force 3 cycles", lambda: bf.test_bruteforce_12bit_inputs_multicycle(0)),
]


def _load(monkeypatch, path):
    monkeypatch.setattr(oracle, "_SO", path)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: path)


def _compile(src: str, path: str):
    c = path[:-3] + ".c"
    with open(c, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", path, c])


def _failing_pins() -> list:
    failed = []
    for name, pin in PINS:
        try:
            pin()
        except AssertionError:
            failed.append(name)
    return failed


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    path = str(tmp_path / "control.so")
    _compile(open(SRC).read(), path)
    _load(monkeypatch, path)
    assert _failing_pins() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    path = str(tmp_path / "mutant.so")
    _compile(src.replace(old, new), path)
    _load(monkeypatch, path)
    assert _failing_pins(), "no pin catches: " + name

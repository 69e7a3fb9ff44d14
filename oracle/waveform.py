"""Waveform events from per-cycle traces -- TEST INFRASTRUCTURE ONLY.

Sec. 6.2 ("Waveform Generation"): record a signal's value when it changes,
detected by comparing each signal's value with its value in the previous
cycle.  Given the probed values before a step and the end-of-cycle trace of
the step, this lists every (cycle, probe, instance, value) whose value differs
from the previous cycle's (cycle 0: from the value before the step).
"""
from __future__ import annotations

import numpy as np


def changes(before: np.ndarray, trace: np.ndarray, cycles) -> np.ndarray:
    """before: [n_probe][n_inst]; trace: [n_cycles][n_probe][n_inst]; cycles: per-instance
    cycle counts (rows past an instance's count are ignored).  Returns an int64 array
    [n_events][4] of (cycle, probe, instance, value) sorted lexicographically."""
    n_cyc, n_probe, n_inst = trace.shape
    cyc = np.broadcast_to(np.asarray(cycles, np.int64), (n_inst,))
    out = []
    for i in range(n_inst):
        prev = before[:, i].copy()
        for c in range(int(cyc[i])):
            cur = trace[c, :, i]
            for p in np.nonzero(cur != prev)[0]:
                out.append((c, int(p), i, int(cur[p])))
            prev = cur
    if not out:
        return np.zeros((0, 4), np.uint64)
    return np.array(sorted(out), dtype=np.uint64)

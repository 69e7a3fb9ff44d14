"""Each step visits only the live prefix of the lanes (Alg. 1's iterative rank
applied to cycles, per instance): lanes are ordered by expected cycle count, so
instances that have run out of cycles gather at the end, and a launch spans
the lanes up to the last one with cycles left, rounded up to whole warps of
lane chunks.  4,096 instances with uneven budgets are stepped 8 cycles at a
time until all are done; the span reported after each step must be exactly
that prefix, the grid must shrink with it, and sampled instances -- the last
live lane of several steps, the first lane past the boundary, the shortest and
the longest -- must equal the oracle bit for bit (a frozen instance is never
written again)."""
import numpy as np
import pytest

import synth
from synth import DesignSpec
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu

N = 4096


def lane_order(budgets: np.ndarray) -> np.ndarray:
    """Instance of every lane: descending expected cycles, ties in instance order."""
    return np.argsort(-budgets.astype(np.int64), kind="stable")


@pytest.mark.parametrize("kernel,V,gran", [("grid", 8, 256), ("grid", 2, 64), ("stream", 4, None),
                                           ("layer", 2, 64)])
def test_span_follows_live_lanes(kernel, V, gran):
    nl = synth.generate(DesignSpec(n_ops=2500, n_regs=96, depth=14, n_inputs=6, seed=31,
                                   input_widths=(8, 32, 1, 64, 16, 3), n_mems=2, mem_words=16))
    budgets = synth.cycle_budgets(31, N, 4, 70)
    lanes = lane_order(budgets)
    # boundary lanes of a few step counts, plus the extremes
    sample = {int(np.argmin(budgets)), int(np.argmax(budgets)), int(lanes[0]), int(lanes[-1])}
    for k in (2, 4, 6):
        live = int((budgets > 8 * k).sum())
        sample.update({int(lanes[live - 1]), int(lanes[min(live, N - 1)])})
    sample = sorted(sample)
    kw = {"lanes_per_thread": V} if kernel != "stream" else {}
    p = Pair(nl, N, kernel=kernel, seed=31, expected_cycles=budgets, oracle_instances=sample, **kw)
    p.step(1, reset=True, threads=4)
    full_grid = p.sim.info["grid"]
    remaining = budgets.astype(np.int64).copy()
    spans = []
    while remaining.max() > 0:
        per = np.minimum(remaining, 8).astype(np.uint32)
        p.step(per, threads=4)
        remaining -= per
        info = p.sim.info
        live = int((per > 0).sum())
        if kernel == "stream":   # whole chunks of lanes (a multiple of 128 dividing the lanes)
            assert info["last_span"] >= live and info["last_span"] % 128 == 0
        else:
            exp = min(N, -(-live // gran) * gran)
            assert info["last_span"] == exp, (live, info["last_span"], exp)
            if kernel == "grid":
                assert info["last_grid"] <= full_grid
        spans.append(info["last_span"])
    assert spans[-1] < spans[0]                       # the span shrank as instances finished
    assert all(a >= b for a, b in zip(spans, spans[1:]))
    if kernel == "grid" and V == 8:
        assert p.sim.info["last_grid"] < full_grid     # and so did the grid of the last steps
    p.compare()
    p.close()

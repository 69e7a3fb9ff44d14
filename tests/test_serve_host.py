"""Serving policy on the host (no GPU): lane allocation, admission by memory
footprint, continuous batching, completion and latency bookkeeping, checked
with a bookkeeping stand-in for the simulation."""
import numpy as np
import pytest

from paper_2601_18140_gb300.serve import Job, LaneRanges, Server, latency_stats, poisson_trace


class FakeSim:
    """Counts, per lane, the cycles run and the reset cycles since the last lane reset."""
    created = []

    def __init__(self, name, cap):
        self.name, self.cap = name, cap
        self.cycles = np.zeros(cap, np.int64)
        self.resets = np.zeros(cap, np.int64)
        self.seed = np.zeros(cap, np.int64)
        self.steps = 0
        self.closed = False
        FakeSim.created.append(self)

    def reset_lanes(self, b, n, seeds):
        self.cycles[b:b + n] = 0
        self.resets[b:b + n] = 0
        self.seed[b:b + n] = -1 if seeds is None else seeds[0, 0]

    def step(self, per, stimulus, reset_per_instance):
        self.steps += 1
        per = np.asarray(per, np.int64)
        self.resets += np.minimum(per, np.asarray(reset_per_instance, np.int64))
        self.cycles += per

    def sync(self):
        pass

    def read(self, signals, b, n):
        return np.stack([self.cycles[b:b + n], self.resets[b:b + n], self.seed[b:b + n]])

    def close(self):
        self.closed = True


def make(capacity, budget, quantum=10, fp=100):
    return Server(lambda name, cap: FakeSim(name, cap), lambda name, cap: fp * cap,
                  {"a": 1, "b": 1}, {"a": 1, "b": 1}, {"a": [0], "b": [0]}, capacity, budget,
                  quantum, seeds=lambda job: np.full((1, job.n_instances), job.seed))


def test_lane_ranges_first_fit_and_merge():
    lr = LaneRanges(10)
    a, b, c = lr.alloc(3), lr.alloc(3), lr.alloc(3)
    assert (a, b, c) == (0, 3, 6) and lr.alloc(2) is None
    lr.release(3, 3)
    assert lr.alloc(4) is None and lr.alloc(3) == 3
    lr.release(0, 3)
    lr.release(3, 3)
    lr.release(6, 3)
    assert lr.free == [[0, 10]]


def test_every_job_runs_exactly_its_cycles_after_one_reset():
    srv = make({"a": 16, "b": 8}, budget=10_000)
    jobs = [Job(k, "ab"[k % 2], 1 + k % 5, 3 + 7 * k, seed=100 + k, arrival=0.0) for k in range(12)]
    done = srv.run(jobs)
    assert len(done) == 12
    for j in done:
        cyc, rst, seed = j.result
        assert (cyc == j.cycles + 1).all() and (rst == 1).all() and (seed == j.seed).all()
        assert j.admitted is not None and j.finished >= j.admitted


def test_continuous_batching_shares_launches():
    """Jobs admitted at different rounds advance in the same launches."""
    srv = make({"a": 64, "b": 8}, budget=10_000, quantum=5)
    jobs = [Job(0, "a", 4, 50, 1), Job(1, "a", 4, 10, 2), Job(2, "a", 8, 30, 3)]
    done = srv.run(jobs)
    assert len(done) == 3
    sim = FakeSim.created[-1]
    assert sim.steps == srv.rounds == 11      # ceil(51 / 5): one launch per round for all jobs
    assert {j.job_id for j in done[:1]} == {1}                     # the short job finishes first


def test_admission_by_footprint_and_idle_pool_release():
    FakeSim.created.clear()
    # each pool costs 100 * capacity; the budget holds one pool at a time
    srv = make({"a": 10, "b": 10}, budget=1_500)
    jobs = [Job(0, "a", 5, 20, 1), Job(1, "b", 5, 20, 2), Job(2, "a", 5, 5, 3)]
    done = srv.run(jobs)
    assert len(done) == 3
    assert srv.used() <= 1_500
    assert any(s.closed for s in FakeSim.created)            # an idle pool made room
    with pytest.raises(RuntimeError):
        make({"a": 100, "b": 1}, budget=50).run([Job(0, "a", 1, 1, 1)])


def test_queue_waits_for_lanes():
    srv = make({"a": 4, "b": 4}, budget=10_000, quantum=3)
    jobs = [Job(k, "a", 3, 9, k) for k in range(3)]         # only one fits at a time
    done = srv.run(jobs)
    assert [j.job_id for j in done] == [0, 1, 2]
    assert done[1].admitted >= done[0].finished - 1e-9


def test_trace_and_stats():
    tr = poisson_trace(4, 200, 100.0, ["a", "b", "c"], np.log(1e4), 1.0, 64, cycles_cap=None)
    assert len(tr) == 200 and all(1 <= j.n_instances <= 64 for j in tr)
    arr = np.array([j.arrival for j in tr])
    assert (np.diff(arr) > 0).all() and 1.0 < arr[-1] < 3.5            # ~200 / 100 Hz
    cyc = np.array([j.cycles for j in tr])
    assert 5_000 < np.median(cyc) < 20_000                             # median e^mu = 10k
    for k, j in enumerate(tr[:10]):
        j.arrival, j.finished = 0.0, float(k)
    s = latency_stats(tr[:10])
    assert s["n"] == 10 and s["p50_s"] == pytest.approx(4.5) and s["max_s"] == 9.0

"""Host-side pieces of the benchmark: the workloads are the configurations they
claim to be, the algorithmic byte count follows its definition on a hand-built
circuit, shards cover every instance exactly once, and DRAM records apply only
to the kernel sources they were taken on."""
import os

import numpy as np

import bench
import synth
from synth import Builder


def test_workload_sizes():
    spec = synth.spec_batch()
    assert (spec.n_ops, spec.n_regs, spec.depth, spec.n_inputs) == (1_000_000, 65_536, 80, 32)
    assert bench.WORKLOADS["batch-1M"][1] == 4096 and bench.WORKLOADS["batch-1M"][2] == (1000, 100_000)
    spec = synth.spec_soc()
    assert (spec.n_ops, spec.n_regs, spec.depth, spec.n_mems, spec.mem_words) == (5_000_000, 262_144, 120, 64, 32)
    assert bench.WORKLOADS["soc-5M"][1] == 1024
    spec = synth.spec_single()
    assert (spec.n_ops, spec.n_regs, spec.depth) == (200_000, 20_000, 60)
    spec = synth.spec_tiny()
    assert (spec.n_ops, spec.n_regs, spec.depth, spec.n_inputs, spec.counter_lfsr) == (2000, 64, 20, 8, True)
    q = synth.spec_quiet()
    assert q.n_modules * q.ops_per_module == 1_000_000
    budgets = synth.cycle_budgets(5, 4096, 1000, 100_000)
    assert budgets.min() >= 1000 and budgets.max() <= 100_000


def test_algorithmic_bytes_on_a_hand_built_circuit():
    b = Builder()
    i = b.input(8)                     # 1 byte per lane
    r = b.reg(32)                      # 4 bytes
    c = b.const(16, 3)                 # 2 bytes
    s = b.op("ADD", 32, r, c)          # reads 4 + 2, writes 4
    t = b.op("MUX", 64, i, s, r)       # reads 1 + 4 + 4, writes 8
    b.connect(r, s)                    # D read 4, Q write 4
    nl = b.build()
    got = bench.algorithmic_bytes_per_instance_cycle(nl, lanes_sharing_meta=4)
    assert got["ops"] == (4 + 2 + 4) + (1 + 4 + 4 + 8)
    assert got["regs"] == 4 + 4
    assert got["inputs"] == 16 + 1     # xorshift state read + written, input row
    assert got["meta"] == 20.0 * 2 / 4
    assert got["total"] == got["ops"] + got["regs"] + got["inputs"] + got["mem"] + got["meta"]
    del t


def test_shards_cover_every_instance_once():
    for n in [1, 7, 4096, 1000]:
        for world in [1, 2, 3, 8]:
            seen = np.zeros(n, np.int64)
            for rank in range(world):
                lo, hi = bench.shard(n, rank, world)
                seen[lo:hi] += 1
            assert (seen == 1).all()


def test_traffic_records_follow_the_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 12 and h == bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("# comment\nk_grid:batch-1M 123 %s\nk_grid:soc-5M 456 0123456789ab\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profile_traffic("k_grid:batch-1M") == 123.0
    assert bench.profile_traffic("k_grid:soc-5M") is None       # taken on other sources
    assert bench.profile_traffic("k_tile:batch-1M") is None


def test_measured_peak_is_read_from_the_driver_file():
    p = bench.measured_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert p["source"] == "measured" and p["hbm_gbs"] > 1000
    else:
        assert p["source"] == "fallback"


def test_live_ops_is_the_cone_of_state():
    """Ops counted live: the fan-in cone of register next states and write-port
    signals; an op read only by a dead op is dead too."""
    b = Builder()
    i = b.input(8)
    r = b.reg(8)
    m = b.mem(4, 8)
    a = b.op("ADD", 8, r, i)            # live: feeds the register through x
    x = b.op("XOR", 8, a, i)            # live: the register's D
    b.op("NOT", 8, x)                   # dead: read by nothing ...
    d2 = b.op("AND", 8, a, i)           # dead: read only by a dead op
    b.op("OR", 8, d2, i)                # dead
    en = b.op("ORR", 1, i)              # live: a write-port enable
    b.connect(r, x)
    b.write_port(m, en, i, r)
    assert bench.live_ops(b.build()) == 3

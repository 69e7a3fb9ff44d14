"""Multi-GPU form = replicas (instances are independent; no exchange step exists
in the cascade): each rank simulates a contiguous shard of the instances, and
the whole-job time is the slowest rank's.  Checked on CPU with two gloo ranks,
the oracle standing in for each rank's device: the shards together reproduce
the single-process result, and the reduction takes max time / summed work."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, cycles, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nl = synth.generate(synth.DesignSpec(n_ops=400, n_regs=30, depth=8, n_inputs=3, seed=33))
    lo, hi = bench.shard(n, rank, world)
    xs = np.ascontiguousarray(synth.xorshift_seeds(33, nl.n_inputs, n)[:, lo:hi])
    o = oracle.OracleSim(nl.to_bytes(), hi - lo)
    o.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    o.step(cycles, mode=oracle.STIM_XORSHIFT, xs=xs)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, o.vals.copy()))
    t_max, evals = bench.reduce_over_ranks(10.0 * (rank + 1), float((hi - lo) * cycles * nl.n_ops), "cpu")
    if rank == 0:
        q.put((parts, t_max, evals))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_reproduce_the_single_run():
    import oracle
    import synth
    n, cycles, world = 13, 17, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, cycles, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts, t_max, evals = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    shards = sorted(parts)
    assert shards[0][0] == 0 and shards[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(shards, shards[1:]))          # contiguous, disjoint
    nl = synth.generate(synth.DesignSpec(n_ops=400, n_regs=30, depth=8, n_inputs=3, seed=33))
    xs = synth.xorshift_seeds(33, nl.n_inputs, n)
    full = oracle.OracleSim(nl.to_bytes(), n)
    full.step(1, reset=True, mode=oracle.STIM_XORSHIFT, xs=xs)
    full.step(cycles, mode=oracle.STIM_XORSHIFT, xs=xs)
    assert np.array_equal(np.concatenate([p[2] for p in shards]), full.vals)
    assert t_max == 20.0                                       # slowest rank
    assert evals == float(n * cycles * nl.n_ops)               # all ranks' work

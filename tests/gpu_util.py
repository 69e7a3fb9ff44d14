"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare every signal, memory word and stimulus state."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2601_18140_gb300 as rt
import synth

MODES = {"hold": oracle.STIM_HOLD, "xorshift": oracle.STIM_XORSHIFT, "buffer": oracle.STIM_BUFFER}


class Pair:
    def __init__(self, nl: synth.Netlist, n_inst: int, kernel="auto", seed: int = 0,
                 expected_cycles=None, oracle_instances=None, fuse_mux_chains: bool = False, **sim_kw):
        self.nl = nl
        self.n = n_inst
        self.xs = synth.xorshift_seeds(seed, nl.n_inputs, n_inst)
        self.design = rt.Design(nl.to_bytes(), fuse_mux_chains=fuse_mux_chains)
        self.sim = rt.Sim(self.design, n_inst, kernel=kernel, xorshift_seed=self.xs,
                          expected_cycles=expected_cycles, **sim_kw)
        # the oracle may follow only a sample of instances (large workloads)
        self.sample = (np.arange(n_inst) if oracle_instances is None
                       else np.asarray(oracle_instances, np.int64))
        self.orc = oracle.OracleSim(nl.to_bytes(), self.sample.size)
        self.oxs = np.ascontiguousarray(self.xs[:, self.sample])

    def step(self, cycles, stimulus="xorshift", reset=False, values=None, probes=None,
             probe_mode="last", threads=8):
        per = None if np.isscalar(cycles) else np.asarray(cycles, np.uint32)
        vals_dev = None
        if values is not None:
            import torch
            vals_dev = torch.from_numpy(np.ascontiguousarray(values)).cuda()
        g = self.sim.step(cycles, stimulus=stimulus, values=vals_dev, reset=reset, probes=probes,
                          probe_mode=probe_mode)
        ocyc = cycles if per is None else per[self.sample]
        obuf = None if values is None else np.ascontiguousarray(values[:, :, self.sample])
        pc = 0
        if probes is not None and probe_mode == "every":
            pc = int(np.max(cycles))
        o = self.orc.step(ocyc, reset=reset, mode=MODES[stimulus], xs=self.oxs, buf=obuf,
                          probes=probes, probe_cycles=pc, threads=threads)
        if probes is not None:
            if probe_mode == "every":
                got = g[:, :, self.sample]
                # rows past an instance's own cycle count are not written by either side
                for k, i in enumerate(self.sample):
                    c = int(ocyc if np.isscalar(ocyc) else ocyc[k])
                    assert np.array_equal(got[:c, :, k], o[:c, :, k]), "probe trace differs"
            else:
                exp = self.orc.read(probes)
                assert np.array_equal(g[:, self.sample], exp), "last-cycle probes differ"

    def compare(self):
        sampled = self.sample.size != self.n
        if sampled:  # read back only the instances the oracle follows
            g = np.concatenate([self.sim.read(None, int(i), 1) for i in self.sample], axis=1)
        else:
            g = self.sim.read()
        exp = self.orc.read()
        if not np.array_equal(g, exp):
            bad = np.argwhere(g != exp)
            sig, k = bad[0]
            raise AssertionError("state differs at %d places; first: signal %d instance %d: "
                                 "gpu %#x oracle %#x" % (len(bad), sig, self.sample[k],
                                                          int(g[sig, k]), int(exp[sig, k])))
        if self.nl.n_mems:
            gm = (np.concatenate([self.sim.read_mem(int(i), 1) for i in self.sample], axis=1)
                  if sampled else self.sim.read_mem())
            assert np.array_equal(gm, self.orc.read_mem())
        if self.nl.n_inputs:
            gx = (np.concatenate([self.sim.read_stim_state(int(i), 1) for i in self.sample], axis=1)
                  if sampled else self.sim.read_stim_state())
            assert np.array_equal(gx, self.oxs)

    def close(self):
        self.sim.close()
        self.design.close()

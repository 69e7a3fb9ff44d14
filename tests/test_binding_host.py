"""The Python binding refuses host buffers of the wrong shape before the library
reads them (the C ABI takes plain pointers and cannot check their sizes).
Runs on the CPU: every check fires before any call into the library."""
import numpy as np
import pytest

import paper_2601_18140_gb300 as rt


class _Design:
    handle = 0
    info = {"n_inputs": 3, "mem_words_total": 8, "n_signals": 10}


def _sim(n=4):
    s = rt.Sim.__new__(rt.Sim)
    s.design, s.n, s.handle = _Design(), n, 0
    return s


def test_sim_creation_checks_per_instance_arrays():
    with pytest.raises(ValueError):
        rt.Sim(_Design(), 4, expected_cycles=np.zeros(3, np.uint32), use_torch_allocator=False)
    with pytest.raises(ValueError):
        rt.Sim(_Design(), 4, xorshift_seed=np.ones((3, 5), np.uint64), use_torch_allocator=False)


def test_state_memory_and_stimulus_buffers():
    s = _sim()
    with pytest.raises(ValueError):
        s.write_mem(np.zeros((7, 4), np.uint64))            # rows must be mem_words_total
    with pytest.raises(ValueError):
        s.write_stim_state(np.zeros((2, 4), np.uint64))     # rows must be n_inputs
    with pytest.raises(ValueError):
        s.reset_lanes(0, 2, np.ones((3, 3), np.uint64))     # [n_inputs][n_inst]
    with pytest.raises(ValueError):
        s.write([0, 1], np.zeros((3, 4), np.uint64))        # one row per signal
    with pytest.raises(ValueError):                         # [cycles][n_inputs][n_instances]
        s.step(5, stimulus="buffer", values=np.zeros((4, 3, 4), np.uint64))
    with pytest.raises(ValueError):
        s.step(np.ones(3, np.uint32))                       # one budget per instance
    with pytest.raises(ValueError):
        s.step(2, reset_per_instance=np.ones(5, np.uint32))

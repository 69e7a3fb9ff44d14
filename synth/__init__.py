"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

Holds the netlist container / serialiser and the seeded generators for
designs, stimulus seeds and cycle budgets.  It contains none of the
simulation arithmetic: nothing here evaluates an operation.
"""
from .netlist import ARITY, MAGIC, N_OPCODES, OP, OPNAME, VERSION, Builder, Netlist
from .gen import (GEN_VERSION, DesignSpec, Rng, cycle_budgets, generate, spec_batch,
                  spec_mux, spec_quiet, spec_serving, spec_single, spec_soc, spec_tiny, splitmix64_mix,
                  ModularSpec, generate_modular,
                  stimulus_values, xorshift_seeds)

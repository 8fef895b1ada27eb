"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws inputs: one- and two-electron integrals shaped like the
paper's active spaces, occupation vectors of determinants, and random
block-sparse MPS site tensors.  It contains none of the method's arithmetic (no
Hamiltonian action, no fitting, no time stepping), so both the CPU oracle and
the CUDA path may read from it without sharing any of the computation.
"""
from .integrals import make_integrals, IntegralSet
from .states import (aufbau_occupation, hole_occupation, occupation_charge,
                     random_mps, bond_sectors)

__all__ = ["make_integrals", "IntegralSet", "aufbau_occupation",
           "hole_occupation", "occupation_charge", "random_mps", "bond_sectors"]

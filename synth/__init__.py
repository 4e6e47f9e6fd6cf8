"""Seeded synthetic inputs for the ppRPA hot path.

This module only draws random numbers and arranges them into the input set
that a mean-field code would hand to ppRPA (occupation numbers, orbital
energies, MO coefficients and three-center density-fitting integrals).
It holds none of the ppRPA arithmetic, so both the CPU oracle and the GPU
harness can use it without sharing any method code.
"""
from .generators import (  # noqa: F401
    SystemSpec,
    CONFIGS,
    make_system,
    ao_slices,
    batch_molecule_spec,
    random_trial_vectors,
)

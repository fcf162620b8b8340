"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds no arithmetic of the molecular-dynamics method itself: it only
draws the initial conditions (lattice sites, species labels, Maxwell-Boltzmann
velocities, random non-overlapping positions) from a counter-based generator whose
definition is given in :mod:`inputs.generate`.
"""
from .generate import (  # noqa: F401
    GAMMA,
    splitmix64,
    counter_u64,
    uniform01,
    gaussian,
    fcc_lattice,
    box_for,
    assign_species,
    maxwell_boltzmann,
    rsa_positions,
    Workload,
    workload,
    STREAM_SPECIES,
    STREAM_VEL,
    STREAM_RSA,
)

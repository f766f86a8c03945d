"""Seeded synthetic QM/MM inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random geometry, basis exponents/coefficients, MM charges and density
matrices; it holds none of the method's arithmetic (no normalisation, integrals or Ewald sums).
Every generator is deterministic in its seed (numpy PCG64).

The workloads stand in for the paper's systems (QM water in MM water, Sec. "QM Water in MM
Water"; enzyme active sites, Secs. "Guanosine Triphosphate Hydrolysis" and "Chorismate Mutase"),
whose coordinates are not available: MM water is rigid TIP3P geometry on a jittered lattice, the
QM region a cluster of atoms with a seeded contracted Cartesian basis.
"""
from .synth import (  # noqa: F401
    ANGSTROM_TO_BOHR,
    System,
    config1_water,
    config2_active_site,
    config4_large_site,
    config5_frames,
    make_cluster_system,
    random_density,
    small_system,
    SEED_BASE,
)

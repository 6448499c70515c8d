"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This package only *draws* inputs: random SU(3) fields, the synthetic fat (X) and Naik (N)
links with the staggered phases and the fermion boundary signs folded in, Gaussian and Z2
right-hand sides, and random gauge transforms.  It holds none of the Dslash, operator or
solver arithmetic; neither the oracle nor the CUDA library is imported here.
"""
from .gauge import (  # noqa: F401
    SEED_FAT_U, SEED_FAT_NOISE, SEED_NAIK_U, SEED_RHS_BASE, SEED_GAUGE_TRANSFORM,
    Lattice, random_su3, fat_links, naik_links, free_field_links, gaussian_rhs, z2_rhs,
    gauge_transform_field, staggered_phases, boundary_signs, even_odd_embed,
)

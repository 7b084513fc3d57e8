"""Seeded synthetic inputs for the environment-potential path.

This module only builds inputs: point charges, Gaussian primitive pairs with
density weights, and electron positions.  It holds none of the potential
arithmetic (no Boys function, no Hermite expansion, no Coulomb integral), so
both the CPU oracle and the CUDA library can consume what it produces without
sharing any of the method's code.

Units are bohr, hartree and elementary charge.  The QM region is a sphere of
radius 6 bohr about the origin; environment charges sit outside it, as in the
paper's QM/MM split of the glycine trimer (Sec. II.B, Eq. ElectrostaticField:
nuclei {Z_beta, R_beta} plus the density of the other fragments).
"""
from .generate import (  # noqa: F401
    PairList,
    Workload,
    qm_positions,
    small_environment,
    realistic_environment,
    batched_environments,
    batched_specs,
    batched_system,
    tiny_pd_environment,
    point_cells_environment,
    seed_for_config,
)

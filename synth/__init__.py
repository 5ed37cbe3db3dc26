"""Seeded synthetic inputs for the Newton-step linear solve.

This package produces *inputs* only: meshes, per-element Hessian blocks
(row, col, 3x3) triplets, contact pairs, the mesh adjacency graph and
right-hand sides.  It contains none of the solver's arithmetic (no
assembly, partition, MAS or PCG), so both the CUDA path and the oracle can
consume its output without sharing method code.

The workloads stand in for the paper's scenes (octopus, bunnies, cloth,
...), which are not available: unit tet cubes split 5 tets per cell with a
stable Neo-Hookean Hessian, lumped mass / dt^2, and random PSD contact
blocks.
"""

from .mesh import tet_cube, tet_edges, adjacency_csr  # noqa: F401
from .hessians import (  # noqa: F401
    snh_element_blocks,
    lumped_mass_blocks,
    contact_blocks,
    random_pairs,
    near_pairs,
)
from .workloads import make_tet_system, make_tet_systems, TetSystem, rhs  # noqa: F401

"""Seeded synthetic inputs for the DEC steady-conduction path.

This package holds input generation only: lattices, the Delaunay mesher,
conductivity fields, penny-shaped discs, boundary tags and Dirichlet values.
It contains none of the method's arithmetic (no Hodge star, no Laplacian, no
solver) and is shared, unchanged, by the CPU oracle and the CUDA path so that
both see byte-identical inputs.

The paper meshes a unit cube with TetGen (Sec. 3.1, 3.2) and studies a cube
with Dirichlet temperatures 1 and 0 on two opposite faces and insulated
remaining faces (Sec. 2.5); the synthetic meshes here stand in for those
TetGen meshes.
"""
from .mesh import (kuhn_lattice, jittered_lattice, delaunay_lattice,
                   canonical_tets, lattice_spacing)
from .fields import (node_tags, dirichlet_values, lognormal_conductivity,
                     conductivity_fields, penny_discs, crack_scales, FREE,
                     DIRICHLET, NEUMANN)
from .workloads import Workload, make_workload, make_fields, WORKLOADS

__all__ = [
    "kuhn_lattice", "jittered_lattice", "delaunay_lattice", "canonical_tets",
    "lattice_spacing", "node_tags", "dirichlet_values",
    "lognormal_conductivity", "conductivity_fields", "penny_discs",
    "crack_scales", "FREE", "DIRICHLET", "NEUMANN", "Workload",
    "make_workload", "make_fields", "WORKLOADS",
]

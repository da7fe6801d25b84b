"""Seeded synthetic inputs for the MOREA objective evaluator.

This package only *generates* inputs (images, meshes, solutions, partial-move
requests).  It holds none of the method's arithmetic: no snapping, no
orientation tests, no rasterisation, no sampling and no objective.  Both the
CUDA path (through its binding) and the CPU oracle consume what it produces.
"""

from .phantom import (  # noqa: F401
    Problem,
    make_problem,
    make_c0,
    make_c1,
    make_c2,
    make_c4,
    kuhn_lattice,
    label_pair,
    lattice_points,
    jitter_population,
    partial_requests,
    vertex_adjacency,
    CONFIGS,
)

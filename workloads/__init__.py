"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This package builds meshes (vertex coordinates and P1 simplex connectivity),
initial states, stimulus node sets and batch-instance parameters.  It holds no
arithmetic of the method itself: no assembly, no quadrature, no ionic model and
no time stepping.  Both the CUDA library and the CPU oracle receive the arrays
it produces, so neither depends on the other.
"""

from .meshes import (  # noqa: F401
    Mesh,
    grid2d,
    kuhn3d,
    ventricle_shell,
)
from .configs import (  # noqa: F401
    Workload,
    w0_square,
    w1_slab,
    w1l_slab,
    w4_slab,
    w5_tissue,
    tiny,
    batch_instances,
    AP_BENCH,
    AP_PAPER,
    SEED_BASE,
)

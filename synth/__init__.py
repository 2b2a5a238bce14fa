"""Seeded synthetic inputs shared by the tests, the bench and the smoke run.

This module holds no arithmetic of the solver: it only draws design fields and
writes load vectors.  Both the CUDA path and the CPU oracle consume what it
produces; neither is imported here.

Mesh conventions (shared by every input):
  * nelx x nely unit-square elements; element e = j*nelx + i.
  * nodes (nelx+1) x (nely+1), node n = j*(nelx+1) + i, x index fastest.
  * DOF 2n is u_x, DOF 2n+1 is u_y, so a nodal vector is laid out
    [nely+1][nelx+1][2].
  * Design fractions are laid out [n_phase][nely][nelx].
"""

from .designs import (  # noqa: F401
    BOTTOM,
    LEFT,
    RIGHT,
    TOP,
    batch_sizes,
    dirichlet_design,
    dirichlet_design_torch,
    load_right_edge,
    load_top_edge,
    splitmix64,
    uniform01,
)

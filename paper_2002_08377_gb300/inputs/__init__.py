"""Seeded synthetic inputs: Voronoi meshes, angle sets and the five workloads.

This module holds no arithmetic of the radiation method.  It builds the
host arrays that both the CPU oracle and the CUDA path take as input:
generator points (numpy default_rng), the periodic Voronoi tessellation
(native builder in voronoi.cpp), the level-symmetric angle sets and the
per-cell gas / boundary / emitter fields of the paper's test problems
(Sec. 3) at the sizes of the synthetic workloads.
"""
from .mesh import Mesh, build_mesh, jittered_lattice, build_voronoi_lib  # noqa: F401
from .angles import level_symmetric, n_angles  # noqa: F401
from .workloads import (Problem, make_problem, WORKLOADS, thermal, shadows, diffusion,  # noqa: F401
                        adjoint, waves, KIND_INTERIOR, KIND_BOUNDARY, KIND_EMITTER)

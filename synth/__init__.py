"""Seeded synthetic dynamic-mesh sequences.

These generators stand in for the animated meshes the paper evaluates on
(Handstand, Samba, Dinosaur, Chinchilla, Camel-gallop, Flag; Section IV,
Table II), which are not available here.  They produce meshes with fixed
connectivity and a sequence of F frames of vertex positions, with sizes and
motion types of the same kind: smooth articulated/rigid motion, travelling
waves, moving bumps and, where asked, i.i.d. noise.

This module holds no arithmetic of the compression method itself (no
Laplacian, no subspace iteration, no quantizer).  Both the oracle and the
CUDA path consume its outputs; neither is imported here.

Conventions
-----------
* ``tris``      int32 [T, 3], vertex indices, 0-based.
* ``positions`` float64 [F, n, 3], frame-major, the layout the codec accepts
  at its boundary (the paper's sequence A = [M_1; ...; M_k] of Section II,
  each M_f an n x 3 matrix).
"""

from .meshes import icosphere, torus_grid, open_grid, disjoint_union, sub_mesh  # noqa: F401
from .motion import (  # noqa: F401
    SequenceSpec,
    make_sequence,
    sinusoid_rigid_motion,
    CONFIGS,
    config_spec,
)

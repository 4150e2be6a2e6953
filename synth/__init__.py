"""Seeded synthetic inputs: skeleton samples of peg-in-hole-shaped parts and
random rotation sets.

This module holds no arithmetic of the method itself (no densities, no
transforms, no fields); it only draws the inputs that both the CUDA path and
the FP64 oracle consume.  Every generator is a pure function of its seed.

The paper's own test pair (a three-peg / three-hole assembly with zero
clearance, its Fig. 4) is third-party CAD data; these skeletons stand in for
it: rings, axis segments and planar sheets of skeleton points, each point
carrying a ball radius that becomes the Gaussian width sigma.  Closed
triangle meshes of a peg and a holed block (synth.meshes) stand in for the
CAD B-reps of the paper's mesh descriptor (Eq. 2).
"""
from .skeletons import (  # noqa: F401
    Part,
    c1_pair,
    c2_pair,
    c3_pairs,
    c4_pair,
    c5_sessions,
    random_quaternions,
    ring,
    segment,
    sheet,
    mixed_part,
    quaternion_walk,
    translation_walk,
)
from .meshes import box, cylinder, peg_hole_pair, tube  # noqa: F401

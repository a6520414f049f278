"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This package only produces inputs: triangle meshes (FP32 vertices, int32
indices), aspect-angle lists, frequency lists and request mixes. It contains
none of the scattering arithmetic, so the CUDA path and the CPU oracle can both
consume it without sharing any of the method's code.
"""
from .meshes import icosphere, trihedral, square_plate, dihedral, aircraft, mesh_bbox  # noqa: F401
from .workloads import (  # noqa: F401
    C0, spacing_for, grid_offset, sphere_case, trihedral_case, aircraft_case, batched_requests,
    surrogate_samples,
)

"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds input generators only: unit-cell surface meshes, lattice
descriptions of the benchmark workloads, incidence directions and a PCG32
random stream.  It contains none of the boundary element or fast multipole
arithmetic, so that the CPU oracle and the GPU library can both draw the same
inputs without sharing any of the method's code.
"""
from .meshes import icosphere, capped_cylinder, cube, open_cylinder, quad9_sphere, mesh_signed_volume
from .rng import PCG32, random_complex_vectors
from .configs import WORKLOADS, Workload, fibonacci_directions, SPEED_OF_SOUND, serving_stream

__all__ = [
    "icosphere", "capped_cylinder", "cube", "open_cylinder", "quad9_sphere", "mesh_signed_volume",
    "PCG32", "random_complex_vectors",
    "WORKLOADS", "Workload", "fibonacci_directions", "SPEED_OF_SOUND", "serving_stream",
]

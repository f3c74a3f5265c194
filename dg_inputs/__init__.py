"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only input generation: meshes (vertex coordinates, element
connectivity, boundary tags), seeded random vectors and closed-form data
functions. It contains none of the discretisation's arithmetic, so both the
oracle and the library may import it.
"""
from .mesh import Mesh, jittered_grid, CONFIG_MESHES, config_mesh
from .fields import uniform_field, fourier_rhs_coeffs, manufactured

__all__ = ["Mesh", "jittered_grid", "CONFIG_MESHES", "config_mesh", "uniform_field",
           "fourier_rhs_coeffs", "manufactured"]

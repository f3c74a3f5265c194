"""GB300 (sm_103a) SIPDG pressure-Poisson library: Python binding.

The compute path lives in the C-ABI shared library built from csrc/ (see
include/dg.h). This package only marshals arguments: torch tensors supply
device memory and the current CUDA stream. There is no CPU fallback; if the
library is missing every call raises.
"""
from ._binding import (DG_F32, DG_F64, KERNEL_AUTO, KERNEL_EPT, KERNEL_GEMM, KERNEL_TENSOR, KERNEL_TENSOR_PIPE, KERNEL_TC05, KERNEL_TC64,
                       KERNEL_TILE,
                       InsStepper, TetMesh,
                       PREC_AMG, PREC_INVMASS, PREC_JACOBI, PREC_NONE, PREC_PMG, DgError, Mesh, SolverOpts, default_opts,
                       interpolation_matrix, lib, lib_path, reference_operators)

__all__ = ["Mesh", "TetMesh", "InsStepper", "SolverOpts", "default_opts", "DgError", "DG_F64", "DG_F32", "PREC_NONE", "PREC_JACOBI", "PREC_INVMASS",
           "PREC_PMG", "PREC_AMG", "KERNEL_AUTO", "KERNEL_TILE", "KERNEL_GEMM", "KERNEL_TENSOR", "KERNEL_EPT",
           "KERNEL_TENSOR_PIPE", "KERNEL_TC05", "KERNEL_TC64",
           "reference_operators", "interpolation_matrix", "lib", "lib_path"]

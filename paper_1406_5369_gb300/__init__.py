"""GB300-native geometric multigrid (arXiv:1406.5369 hot path) - Python binding.

The compute path is libmg.so (CUDA kernels for sm_103a behind the C ABI in
include/mg.h, node-based grids, include/mg_cc.h, cell-centred grids, and
include/mg_cd.h, complex diffusion). This package only marshals arguments: PyTorch supplies the
device arena and the stream; every step of every V-cycle runs in the
library's kernels.
"""
from ._capi import (MG_BF16_DC, MG_FIELD_F, MG_FIELD_R, MG_FIELD_U, MG_FP32_DC, MG_FP64,
                    MG_JACOBI, MG_RBGS, MGError, load)
from .solver import Solver, solve_sequence
from .batch import BatchSolver
from .cellgrid import CCSolver
from .cdiff import CDSolver

__all__ = ["Solver", "solve_sequence", "BatchSolver", "CCSolver", "CDSolver", "MGError", "load", "MG_RBGS", "MG_JACOBI", "MG_FP64", "MG_FP32_DC",
           "MG_BF16_DC", "MG_FIELD_U", "MG_FIELD_F", "MG_FIELD_R"]

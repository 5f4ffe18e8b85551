"""GB300 (sm_103a) implementation of the finite-periodic fast multipole BEM
matrix-vector product and its GMRES solve (Jelich, Zhao, Chen, Marburg,
arXiv 2201.12050).

Every step runs in the CUDA library ``libfmpb.so`` (C ABI in
``include/fmpb.h``); this package only marshals arguments.  PyTorch supplies
device memory and streams.
"""
from ._lib import FmpbError, FmpbLibraryMissing, lib
from .api import (Operator, Server, solve_batch, build_blocks, build_blocks_admittance, build_blocks_q9, near2_plan_counts, halfspace_plan,
                  multipole_tables,
                  multipole_tables_admittance, m2l_blocks, circulant_shape,
                  circulant_spectrum, circulant_apply, circulant_apply_bf16, circulant_apply_f32, circulant_apply_static,
                  offset_gemm_bf16, offset_gemm2_bf16, kernel_launches, version,
                  profile_enable, profile_reset, profile_summary, tuning_summary, set_tile_variant, set_dft_plan, FORM_AUTO,
                  FORM_FMM, FORM_PBEM, FORM_FMM2, FP64, FP32, BF16, MIXED, ELEM_TRI3, ELEM_QUAD9)

__all__ = ["Operator", "Server", "solve_batch", "build_blocks", "build_blocks_admittance", "build_blocks_q9", "near2_plan_counts", "halfspace_plan",
           "multipole_tables",
           "multipole_tables_admittance", "m2l_blocks", "circulant_shape",
           "circulant_spectrum", "circulant_apply", "circulant_apply_bf16", "circulant_apply_f32",
           "circulant_apply_static", "offset_gemm_bf16", "offset_gemm2_bf16", "kernel_launches", "version",
           "profile_enable", "profile_reset", "tuning_summary", "set_tile_variant", "set_dft_plan", "profile_summary", "FmpbError",
           "FmpbLibraryMissing", "lib",
           "FORM_AUTO", "FORM_FMM", "FORM_PBEM", "FORM_FMM2", "FP64", "FP32", "BF16", "MIXED", "ELEM_TRI3",
           "ELEM_QUAD9"]

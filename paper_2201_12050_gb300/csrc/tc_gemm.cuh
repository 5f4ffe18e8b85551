// Offset-indexed complex block products on the tensor cores (tc_gemm.cu).
#pragma once
#include <cuda_bf16.h>

#include <string>

#include "common.cuh"

namespace fmpb {

// Up to 3^3 cell offsets per product (the near stencil of a 3-D lattice).
constexpr int TC_MAX_OFF = 27;
struct TcOffsets {
  int n;
  int d[TC_MAX_OFF][3];
};

// Operators of one batched launch: their realified tables (same shapes), the
// columns of operator o following those of o - 1 in X and y.
constexpr int TC_MAX_BATCH = 16;
struct TcBatch {
  int n;
  int64_t tiles;   // column tiles per operator (set at launch)
  const __nv_bfloat16* A[TC_MAX_BATCH];
  int blk[TC_MAX_BATCH];   // operator q's column block in X and y (q itself unless a subset runs)
  int nblk;                // column blocks in X and y
  int64_t kx;              // values of a row of X that hold data (2 k); the rest of its depth reads as zero
};

// Shapes of the realified operands of a complex m x k block.
//   Mp = 2 m rounded up to 128 (tile rows), Kp = 2 k rounded up to 64 (tile depth).
inline int64_t tc_rows(int64_t m) { return (2 * m + 127) / 128 * 128; }
inline int64_t tc_depth(int64_t k) { return (2 * k + 63) / 64 * 64; }

// A (n_off x Mp x Kp BF16) from n_off complex blocks (m x k each), as the
// real matrix of the complex product with rows and columns interleaved:
//   A[2i][2j] = Re T_ij, A[2i][2j+1] = -Im T_ij, A[2i+1][2j] = Im T_ij, A[2i+1][2j+1] = Re T_ij,
// zero outside 2m x 2k.  Values are rounded FP64 -> FP32 -> BF16, each to nearest even.
fmpb_status tc_realify(const cd* T, int n_off, int64_t m, int64_t k, __nv_bfloat16* A, cudaStream_t st);

// X (rows x Kp BF16): row rho holds (Re x_rho0, Im x_rho0, Re x_rho1, ...) of
// the complex row x + rho k, zero-padded to Kp; same rounding as tc_realify.
fmpb_status tc_rows_to_bf16(const cd* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st);

// y[(r Nc + c) m + i] (+)= sum_o sum_j T_o[i][j] x[(r Nc + c - delta_o) k + j]
// for every right-hand side r < R and cell c of the M[0] x M[1] x M[2] grid;
// source cells c - delta_o outside the grid contribute nothing.  A and X as
// produced by tc_realify / tc_rows_to_bf16; FP32 accumulation in tensor
// memory; y complex double.  err: device word, set non-zero (never cleared
// here) if a wait inside the kernel gave up.
fmpb_status tc_offset_gemm(const __nv_bfloat16* A, const TcOffsets& offs, int64_t m, int64_t k, const int M[3], int R,
                           const __nv_bfloat16* X, cd* y, bool accumulate, unsigned* err, cudaStream_t st);
// The same for n_ops operators with tables A[o] of one shape in one launch:
// X and y hold the R Nc columns of operator 0, then those of operator 1, ...
// blk (may be null): the column block of each listed operator, for a subset
// of the operators whose columns X and y hold (null: 0, 1, ..., n_ops - 1).
// A2 (may be null): a tail product added in the same accumulator, per
// operator A2[o] (tc_rows(m) x tc_depth(k2), offset zero) times X2 (rows of
// depth tc_depth(k2), laid out as X): y (+)= sum_o T_o x_{c - delta_o} + T2 x2_c.
// y_f32: y holds complex FP32 (float2) values instead of complex double.
fmpb_status tc_offset_gemm_batch(const __nv_bfloat16* const* A, int n_ops, const TcOffsets& offs, int64_t m,
                                 int64_t k, const int M[3], int R, const __nv_bfloat16* X, void* y, bool accumulate,
                                 unsigned* err, cudaStream_t st, const int* blk = nullptr,
                                 const __nv_bfloat16* const* A2 = nullptr, int64_t k2 = 0,
                                 const __nv_bfloat16* X2 = nullptr, bool y_f32 = false);

// Float-float sources (float4 per complex value: re_hi, re_lo, im_hi, im_lo),
// rounded (hi + lo) -> FP32 -> BF16.
fmpb_status tc_realify_ff(const float4* T, int n_off, int64_t m, int64_t k, __nv_bfloat16* A, cudaStream_t st);
fmpb_status tc_rows_from_ff(const float4* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st);
// Complex FP32 sources (float2 per value), rounded FP32 -> BF16.
fmpb_status tc_rows_from_f32(const float2* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st);

// Per-frequency products Y_f = Lambda_f X_f of the circulant engine for F
// frequencies: A (F x tc_rows(B) x tc_depth(B), from tc_realify_ff of the
// spectrum), X (F R x tc_depth(B) rows, row f R + r), Y [f][r][b] as
// float-float (float4, hi = FP32 accumulator, lo = 0) or, with y_f32, as
// complex FP32 (float2).
fmpb_status tc_freq_gemm(const __nv_bfloat16* A, int64_t F, int64_t B, int R, const __nv_bfloat16* X, void* Y,
                         unsigned* err, cudaStream_t st, bool y_f32 = false);
// The same for n_ops spectra of one shape in one launch: at each frequency
// f, X and Y hold the R rows of operator 0, then those of operator 1, ...
// (F n_ops R rows in all).
fmpb_status tc_freq_gemm_batch(const __nv_bfloat16* const* A, int n_ops, int64_t F, int64_t B, int R,
                               const __nv_bfloat16* X, void* Y, unsigned* err, cudaStream_t st, bool y_f32 = false,
                               const int* blk = nullptr, int n_blocks = 0);

// JSON list of the tile variants the offset-GEMM autotuner chose so far.
fmpb_status tc_tuning_summary(std::string& out);
// Forces tile variant v (0..3) of the offset GEMM, or autotuning (-1).
fmpb_status tc_force_variant(int v);

}  // namespace fmpb

// Device GMRES driver (gmres.cu).
#pragma once
#include <functional>

#include "common.cuh"

namespace fmpb {

// y = A x for R stacked vectors of length N on stream st.
typedef std::function<fmpb_status(int R, const cd* x, cd* y, cudaStream_t st)> MatvecFn;
// The same product on float-float vectors (float4 per value), where the
// operator has one; it saves the conversions around every Arnoldi product.
typedef std::function<fmpb_status(int R, const float4* x, float4* y, cudaStream_t st)> MatvecFfFn;

// The same product on complex FP32 vectors (float2 per value), for operators
// whose products carry BF16 rounding: with it the Krylov basis is FP32.
typedef std::function<fmpb_status(int R, const float2* x, float2* y, cudaStream_t st)> MatvecF32Fn;

// active_host (host, R entries, may be null): kept equal to the systems
// still iterating as of the last poll of the convergence flags (all 1 around
// the restart and true-residual products), so that a caller's product may
// skip systems that have stopped.
// Basis and Gram-Schmidt: A32 given, an FP32 basis with delayed
// reorthogonalisation (DCGS2) on A32's products; else Aff given, a
// float-float basis with DCGS2 on Aff's; else a float-float basis with
// classical Gram-Schmidt and a conditional second pass on A's products.
fmpb_status gmres_solve(const MatvecFn& A, int R, int64_t N, const cd* b, cd* x, const fmpb_solve_opts& o,
                        fmpb_solve_info* info, cudaStream_t st, const MatvecFfFn* Aff = nullptr,
                        int* active_host = nullptr, const MatvecF32Fn* A32 = nullptr);
// GMRES-IR: accurate residuals with A, corrections by GMRES with Alow (on
// FP32 vectors with an FP32 basis when Alow32 is given).
fmpb_status gmres_refined(const MatvecFn& A, const MatvecFn& Alow, int R, int64_t N, const cd* b, cd* x,
                          const fmpb_solve_opts& o, fmpb_solve_info* info, cudaStream_t st,
                          const MatvecF32Fn* Alow32 = nullptr);

}  // namespace fmpb

// Multipole operators (multipole.cu).
#pragma once
#include "common.cuh"
#include "internal.cuh"

namespace fmpb {

constexpr int MAX_NT = 20;   // largest truncation number (B = 441)

// q = n(n+1) + m  ->  (n, m)
__host__ __device__ __forceinline__ void q_to_nm(int q, int& n, int& m) {
  n = (int)sqrt((double)q);
  while (n * n > q) --n;
  while ((n + 1) * (n + 1) <= q) ++n;
  m = q - n * (n + 1);
}

// beta: uniform normalised admittance (adds i k beta int conj(I) dA to V0).
// centres: device, 3 doubles per element, the expansion centre of each
// element's column of V0 and row of U0 (nullptr: the origin).
// dsign: -1 for the mirrored cell of a nine-node half-space operator (the
// double-layer term of its P2M table changes sign), else 1.
fmpb_status multipole_tables(const DeviceMesh& m, double k, cd beta, int nt, cd* V0, cd* U0, cudaStream_t st,
                             const double* centres = nullptr, double dsign = 1.0);
// K(d_o) for n_d translations; block o written at out + dest[o] B B (dest < 0 skipped).
// regular: the table of Eq. (m2l) with I_l in place of O_l (regular translations).
fmpb_status m2l_blocks(int nt, double k, int n_d, const double* dvecs_host, const int64_t* dest_host, cd* out,
                       cudaStream_t st, bool regular = false);
// Applications with float-float tables (V0: B x n, U0: n x B) and float-float p.
fmpb_status p2m_apply(const float4* V0, int n, int B, int64_t columns, const float4* p, cd* Mom, cudaStream_t st);
fmpb_status l2p_apply(const float4* U0, int n, int B, int64_t columns, const cd* Loc, cd* y, cudaStream_t st);

// FP32 operators: complex FP32 tables and p.
fmpb_status p2m_apply_f32(const float2* V0, int n, int B, int64_t columns, const float2* p, cd* Mom, cudaStream_t st);
fmpb_status l2p_apply_f32(const float2* U0, int n, int B, int64_t columns, const cd* Loc, cd* y, cudaStream_t st);

}  // namespace fmpb

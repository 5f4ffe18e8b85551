// Near-field product of the FMPBEM (Sec. 3.2, Eq. (2dPeriodicFMM)): the
// banded multilevel block Toeplitz matrix S with the 3^d unique blocks
// S_delta (|delta|_inf <= 1) applied as
//   y_c = sum_delta S_delta p_{c - delta}   (cells c - delta inside the grid),
// a shifted-column block GEMM: for every delta the n x n block multiplies the
// n x Nc matrix of cell vectors gathered with offset delta.
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "nearfield.cuh"

namespace fmpb {

constexpr int NT_I = 32;   // output rows per CTA
constexpr int NT_C = 32;   // output cells per CTA
constexpr int NT_J = 16;   // reduction slice

// One CTA: rows i0..i0+31 of cells c0..c0+31 of rhs r; 256 threads, 2x2
// outputs each.
__global__ void k_near_apply(const cd* __restrict__ S, const int* __restrict__ offs, int n_near, int n, int Mx,
                             int My, int Mz, const cd* __restrict__ p, cd* __restrict__ y, int accumulate) {
  __shared__ cd Ss[NT_I][NT_J + 1];
  __shared__ cd Ps[NT_J][NT_C + 1];
  const int r = blockIdx.z;
  const int i0 = blockIdx.y * NT_I;
  const int c0 = blockIdx.x * NT_C;
  const int Nc = Mx * My * Mz;
  const int64_t N = (int64_t)Nc * n;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16
  cd acc[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = mkc(0.0, 0.0);
  const cd* pr = p + (int64_t)r * N;
  for (int o = 0; o < n_near; ++o) {
    const int dx = offs[3 * o], dy = offs[3 * o + 1], dz = offs[3 * o + 2];
    const cd* So = S + (size_t)o * n * n;
    for (int j0 = 0; j0 < n; j0 += NT_J) {
      // S tile: 32 x 16
      for (int e = threadIdx.x; e < NT_I * NT_J; e += blockDim.x) {
        const int ii = e / NT_J, jj = e - ii * NT_J;
        const int i = i0 + ii, j = j0 + jj;
        Ss[ii][jj] = (i < n && j < n) ? So[(size_t)i * n + j] : mkc(0.0, 0.0);
      }
      // P tile: 16 x 32, column = source cell c - delta of output cell c
      for (int e = threadIdx.x; e < NT_J * NT_C; e += blockDim.x) {
        const int cc = e / NT_J, jj = e - cc * NT_J;
        const int c = c0 + cc, j = j0 + jj;
        cd v = mkc(0.0, 0.0);
        if (c < Nc && j < n) {
          const int cx = c % Mx, cy = (c / Mx) % My, cz = c / (Mx * My);
          const int sx = cx - dx, sy = cy - dy, sz = cz - dz;
          if (sx >= 0 && sx < Mx && sy >= 0 && sy < My && sz >= 0 && sz < Mz)
            v = pr[((int64_t)(sz * My + sy) * Mx + sx) * n + j];
        }
        Ps[jj][cc] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int jj = 0; jj < NT_J; ++jj) {
        const cd s0 = Ss[ty][jj], s1 = Ss[ty + 16][jj];
        const cd q0 = Ps[jj][tx], q1 = Ps[jj][tx + 16];
        acc[0][0] = cfma(s0, q0, acc[0][0]);
        acc[0][1] = cfma(s0, q1, acc[0][1]);
        acc[1][0] = cfma(s1, q0, acc[1][0]);
        acc[1][1] = cfma(s1, q1, acc[1][1]);
      }
      __syncthreads();
    }
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (i < n && c < Nc) {
        cd* d = y + (int64_t)r * N + (int64_t)c * n + i;
        *d = accumulate ? cadd(*d, acc[a][b]) : acc[a][b];
      }
    }
}

fmpb_status near_apply(const cd* S, const int* offs_dev, int n_near, int n, const int M[3], int R, const cd* p, cd* y,
                       bool accumulate, cudaStream_t st) {
  const int Nc = M[0] * M[1] * M[2];
  if (R > 65535) {
    set_error("near_apply: too many right-hand sides");
    return FMPB_EINVAL;
  }
  dim3 grid((unsigned)((Nc + NT_C - 1) / NT_C), (unsigned)((n + NT_I - 1) / NT_I), (unsigned)R);
  FMPB_LAUNCH("near_apply", st, k_near_apply<<<grid, 256, 0, st>>>(S, offs_dev, n_near, n, M[0], M[1], M[2], p, y, accumulate ? 1 : 0));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

}  // namespace fmpb

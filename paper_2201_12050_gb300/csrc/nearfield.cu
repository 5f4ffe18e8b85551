// Near-field product of the FMPBEM (Sec. 3.2, Eq. (2dPeriodicFMM)): the
// banded multilevel block Toeplitz matrix S with the 3^d unique blocks
// S_delta (|delta|_inf <= 1) applied as
//   y_c = sum_delta S_delta p_{c - delta}   (cells c - delta inside the grid),
// a shifted-column block GEMM: for every delta the n x n block multiplies the
// n x Nc matrix of cell vectors gathered with offset delta.  The blocks and
// the input are float-float pairs and the products run in float-float
// arithmetic (FP64-class accuracy on the FP32 pipe, which GB300 executes 58
// times faster than FP64).
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "nearfield.cuh"
#include "ff.cuh"

namespace fmpb {

constexpr int NT_I = 32;   // output rows per CTA
constexpr int NT_C = 32;   // output cells per CTA
constexpr int NT_J = 16;   // reduction slice

// One CTA: rows i0..i0+31 of cells c0..c0+31 of rhs r; 256 threads, 2x2
// outputs each.  S (float-float, n_near x n x n) and p (float-float) are
// staged through shared memory; products use float-float arithmetic on the
// FP32 pipe; y is complex double.
__global__ void __launch_bounds__(256) k_near_apply_ff(const float4* __restrict__ S, const int* __restrict__ offs,
                                                       int n_near, int n, int Mx, int My, int Mz,
                                                       const float4* __restrict__ p, cd* __restrict__ y,
                                                       int accumulate) {
  __shared__ float4 Ss[NT_I][NT_J + 1];
  __shared__ float4 Ps[NT_J][NT_C + 1];
  const int r = blockIdx.z;
  const int i0 = blockIdx.y * NT_I;
  const int c0 = blockIdx.x * NT_C;
  const int Nc = Mx * My * Mz;
  const int64_t N = (int64_t)Nc * n;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16
  float rh[2][2], rl[2][2], ih[2][2], il[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) rh[a][b] = rl[a][b] = ih[a][b] = il[a][b] = 0.f;
  const float4* pr = p + (int64_t)r * N;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int o = 0; o < n_near; ++o) {
    const int dx = offs[3 * o], dy = offs[3 * o + 1], dz = offs[3 * o + 2];
    const float4* So = S + (size_t)o * n * n;
    for (int j0 = 0; j0 < n; j0 += NT_J) {
      for (int e = threadIdx.x; e < NT_I * NT_J; e += blockDim.x) {
        const int ii = e / NT_J, jj = e - ii * NT_J;
        const int i = i0 + ii, j = j0 + jj;
        Ss[ii][jj] = (i < n && j < n) ? So[(size_t)i * n + j] : zero;
      }
      // column = source cell c - delta of output cell c
      for (int e = threadIdx.x; e < NT_J * NT_C; e += blockDim.x) {
        const int cc = e / NT_J, jj = e - cc * NT_J;
        const int c = c0 + cc, j = j0 + jj;
        float4 v = zero;
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
        const float4 s0 = Ss[ty][jj], s1 = Ss[ty + 16][jj];
        const float4 q0 = Ps[jj][tx], q1 = Ps[jj][tx + 16];
        ff_cmac(s0, q0, rh[0][0], rl[0][0], ih[0][0], il[0][0]);
        ff_cmac(s0, q1, rh[0][1], rl[0][1], ih[0][1], il[0][1]);
        ff_cmac(s1, q0, rh[1][0], rl[1][0], ih[1][0], il[1][0]);
        ff_cmac(s1, q1, rh[1][1], rl[1][1], ih[1][1], il[1][1]);
      }
      __syncthreads();
    }
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (i < n && c < Nc) {
        cd* d = y + (int64_t)r * N + (int64_t)c * n + i;
        const cd v = mkc((double)rh[a][b] + (double)rl[a][b], (double)ih[a][b] + (double)il[a][b]);
        *d = accumulate ? cadd(*d, v) : v;
      }
    }
}

// FP32 operators: S and p complex FP32 (float2), FP32 FMAs, same tiling.
__global__ void __launch_bounds__(256) k_near_apply_f32(const float2* __restrict__ S, const int* __restrict__ offs,
                                                        int n_near, int n, int Mx, int My, int Mz,
                                                        const float2* __restrict__ p, cd* __restrict__ y,
                                                        int accumulate) {
  __shared__ float2 Ss[NT_I][NT_J + 1];
  __shared__ float2 Ps[NT_J][NT_C + 1];
  const int r = blockIdx.z;
  const int i0 = blockIdx.y * NT_I;
  const int c0 = blockIdx.x * NT_C;
  const int Nc = Mx * My * Mz;
  const int64_t N = (int64_t)Nc * n;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float re[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, im[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  const float2* pr = p + (int64_t)r * N;
  const float2 zero = make_float2(0.f, 0.f);
  for (int o = 0; o < n_near; ++o) {
    const int dx = offs[3 * o], dy = offs[3 * o + 1], dz = offs[3 * o + 2];
    const float2* So = S + (size_t)o * n * n;
    for (int j0 = 0; j0 < n; j0 += NT_J) {
      for (int e = threadIdx.x; e < NT_I * NT_J; e += blockDim.x) {
        const int ii = e / NT_J, jj = e - ii * NT_J;
        const int i = i0 + ii, j = j0 + jj;
        Ss[ii][jj] = (i < n && j < n) ? So[(size_t)i * n + j] : zero;
      }
      for (int e = threadIdx.x; e < NT_J * NT_C; e += blockDim.x) {
        const int cc = e / NT_J, jj = e - cc * NT_J;
        const int c = c0 + cc, j = j0 + jj;
        float2 v = zero;
        if (c < Nc && j < n) {
          const int cx = c % Mx, cy = (c / Mx) % My, cz = c / (Mx * My);
          const int sx = cx - dx, sy = cy - dy, sz = cz - dz;
          if (sx >= 0 && sx < Mx && sy >= 0 && sy < My && sz >= 0 && sz < Mz)
            v = pr[((int64_t)(sz * My + sy) * Mx + sx) * n + j];
        }
        Ps[jj][cc] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int jj = 0; jj < NT_J; ++jj) {
        const float2 s[2] = {Ss[ty][jj], Ss[ty + 16][jj]};
        const float2 q[2] = {Ps[jj][tx], Ps[jj][tx + 16]};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            re[a][b] = fmaf(s[a].x, q[b].x, fmaf(-s[a].y, q[b].y, re[a][b]));
            im[a][b] = fmaf(s[a].x, q[b].y, fmaf(s[a].y, q[b].x, im[a][b]));
          }
      }
      __syncthreads();
    }
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (i < n && c < Nc) {
        cd* d = y + (int64_t)r * N + (int64_t)c * n + i;
        const cd v = mkc((double)re[a][b], (double)im[a][b]);
        *d = accumulate ? cadd(*d, v) : v;
      }
    }
}

fmpb_status near_apply_f32(const float2* S, const int* offs_dev, int n_near, int n, const int M[3], int R,
                           const float2* p, cd* y, bool accumulate, cudaStream_t st) {
  const int Nc = M[0] * M[1] * M[2];
  if (R > 65535) {
    set_error("near_apply: too many right-hand sides");
    return FMPB_EINVAL;
  }
  dim3 grid((unsigned)((Nc + NT_C - 1) / NT_C), (unsigned)((n + NT_I - 1) / NT_I), (unsigned)R);
  FMPB_LAUNCH("near_apply_f32", st, k_near_apply_f32<<<grid, 256, 0, st>>>(S, offs_dev, n_near, n, M[0], M[1], M[2], p, y, accumulate ? 1 : 0));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status near_apply(const float4* S, const int* offs_dev, int n_near, int n, const int M[3], int R, const float4* p,
                       cd* y, bool accumulate, cudaStream_t st) {
  const int Nc = M[0] * M[1] * M[2];
  if (R > 65535) {
    set_error("near_apply: too many right-hand sides");
    return FMPB_EINVAL;
  }
  dim3 grid((unsigned)((Nc + NT_C - 1) / NT_C), (unsigned)((n + NT_I - 1) / NT_I), (unsigned)R);
  FMPB_LAUNCH("near_apply", st, k_near_apply_ff<<<grid, 256, 0, st>>>(S, offs_dev, n_near, n, M[0], M[1], M[2], p, y, accumulate ? 1 : 0));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

}  // namespace fmpb

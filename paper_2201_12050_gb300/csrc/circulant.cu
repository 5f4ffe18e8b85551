// Block Toeplitz products through block circulant embedding and FFT over the
// cell grid (Sec. 2.4, Eqs. (BlockCirculantMatrix), (diagonalized),
// (blockDiagonal), (modifiedFourierTransform1/2); Sec. 3.5, Eq.
// (FMPBEMsystem)).
//
// A multilevel block Toeplitz matrix with blocks T_delta (B x B) is embedded
// in a circulant whose first block column holds T_delta at slot
// (delta mod P) per axis, P >= 2M-1.  Its spectrum is
//   Lambda_f = sum_delta T_delta exp(-2 pi i f.(delta mod P)/P),
// and y = T x is computed as
//   X_f = sum_{c < M} x_c exp(-2 pi i f.c/P)          (pruned forward DFT:
//                                                      only M inputs per axis),
//   Y_f = Lambda_f X_f                               (one B x B product per f),
//   y_c = (1/F) sum_f Y_f exp(+2 pi i f.c/P), c < M   (pruned inverse: only
//                                                      M outputs per axis).
// Grid layout: slot-major, slot f = (fz Py + fy) Px + fx, then R x B (RHS
// outer, coefficient inner); spectrum [f][b][b'] row-major.
//
// Arithmetic: GB300 executes FP64 at 1/58 of its FP32 rate, so for the FP64
// operators every pass (DFTs and block products) runs in float-float
// arithmetic on the FP32 pipe: values are (hi, lo) FP32 pairs carrying 48
// significand bits, products are exact via the fma residual and sums use
// two-sum.  Intermediate grids and the spectrum are then stored as
// float-float (16 bytes per complex value, the size of complex double).  The
// reduced-precision operators keep an FP32 spectrum (SPEC_F32, FP32 passes)
// or a realified BF16 one whose frequency products run on the tensor cores
// (SPEC_BF16; the last forward pass writes their BF16 rows).  Inputs and
// outputs of the product are complex double, or FP32 vectors for the FP32
// Krylov basis.
#include <utility>

#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "ff.cuh"
#include "tc_gemm.cuh"

namespace fmpb {

int padded_length(int M) {
  if (M <= 1) return 1;
  int p = 2 * M - 1;
  for (;; ++p) {
    int q = p;
    for (int f : {2, 3, 5, 7})
      while (q % f == 0) q /= f;
    if (q == 1) return p;
  }
}

CircShape make_shape(const int M[3]) {
  CircShape s;
  s.F = 1;
  s.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    s.M[a] = M[a];
    s.P[a] = padded_length(M[a]);
    s.F *= s.P[a];
    s.ncells *= M[a];
  }
  return s;
}

int64_t offset_slot(const CircShape& s, int dx, int dy, int dz) {
  auto md = [](int d, int P) { return ((d % P) + P) % P; };
  return ((int64_t)md(dz, s.P[2]) * s.P[1] + md(dy, s.P[1])) * s.P[0] + md(dx, s.P[0]);
}

// Direct DFT along one axis for the lines (o1, o2, i), float-float arithmetic:
//   out[o1 b1 + o2 b2 + f bf + i] (+)= scale sum_{j < Pin} in[o1 a1 + o2 a2 + j aj + i] w^{f j},
// w = exp(sign 2 pi i / P), f < Pout.  IN_FF / OUT_FF select float-float
// (float4) or complex-double storage; both are 16 bytes per value, so one
// buffer can change format in place.  A CTA loads one (o1, o2) line group
// for TI consecutive inner indices into shared memory before writing, so the
// call may run in place when in and out use the same strides.
// P1 > 0 selects the two-factor (Cooley-Tukey) form for P = P1 P2: with
// n = P2 n1 + n2 and f = k1 + P1 k2,
//   Y[n2][k1] = w^{n2 k1} sum_{n1} in[P2 n1 + n2] w^{P2 n1 k1}   (P2 DFTs of length P1),
//   out[k1 + P1 k2] = sum_{n2} Y[n2][k1] w^{P1 n2 k2}           (P1 DFTs of length P2),
// P1 Pin + P + Pout P2 products per line instead of Pout Pin.
template <bool IN_FF, bool OUT_FF>
__global__ void k_dft_axis_ff(const void* in_, void* out_, int O2, int64_t I, int64_t a1, int64_t a2, int64_t aj,
                              int64_t b1, int64_t b2, int64_t bf, int Pin, int Pout, int P, int sign, double scale,
                              int accumulate, int TI, int P1) {
  extern __shared__ float4 smf[];
  float4* tw = smf;          // P twiddles (float-float)
  float4* tile = smf + P;    // Pin x TI
  const int o1 = blockIdx.z;
  const int o2 = blockIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * TI;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * j / P, &sn, &cs);
    tw[j] = split_ff(mkc(cs, sign * sn));
  }
  const int64_t base_in = o1 * a1 + o2 * a2 + i0;
  for (int e = threadIdx.x; e < Pin * TI; e += blockDim.x) {
    const int j = e / TI, ii = e - j * TI;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 + ii < I) {
      if (IN_FF)
        v = reinterpret_cast<const float4*>(in_)[base_in + j * aj + ii];
      else
        v = split_ff(reinterpret_cast<const cd*>(in_)[base_in + j * aj + ii]);
    }
    tile[e] = v;
  }
  __syncthreads();
  const int P2 = P1 > 0 ? P / P1 : 0;
  float4* Y = tile + Pin * TI;   // two-factor form: P x TI intermediate values
  if (P1 > 0) {
    for (int e = threadIdx.x; e < P * TI; e += blockDim.x) {
      const int q = e / TI, ii = e - q * TI;   // q = n2 P1 + k1
      const int n2 = q / P1, k1 = q - n2 * P1;
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      const int step = (P2 * k1) % P;
      int idx = 0;
      for (int n = n2; n < Pin; n += P2) {
        ff_cmac(tw[idx], tile[n * TI + ii], rh, rl, ih, il);
        idx += step;
        if (idx >= P) idx -= P;
      }
      float ar = 0.f, al = 0.f, ai = 0.f, ail = 0.f;
      ff_cmac(tw[(n2 * k1) % P], ff_norm(rh, rl, ih, il), ar, al, ai, ail);
      Y[e] = ff_norm(ar, al, ai, ail);
    }
    __syncthreads();
  }
  const int64_t base_out = o1 * b1 + o2 * b2 + i0;
  for (int e = threadIdx.x; e < Pout * TI; e += blockDim.x) {
    const int f = e / TI, ii = e - f * TI;
    if (i0 + ii >= I) continue;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (P1 > 0) {
      const int k1 = f % P1, k2 = f / P1;
      const int step = (P1 * k2) % P;
      int idx = 0;
      for (int n2 = 0; n2 < P2; ++n2) {
        ff_cmac(tw[idx], Y[(n2 * P1 + k1) * TI + ii], rh, rl, ih, il);
        idx += step;
        if (idx >= P) idx -= P;
      }
    } else {
      int idx = 0;
      for (int j = 0; j < Pin; ++j) {
        ff_cmac(tw[idx], tile[j * TI + ii], rh, rl, ih, il);
        idx += f;
        if (idx >= P) idx -= P;
      }
    }
    const int64_t o = base_out + f * bf + ii;
    if (OUT_FF) {
      float4 v = ff_norm(rh, rl, ih, il);
      if (scale != 1.0) {   // float-float product with the float-float scale
        const ff sc = ff_from_d(scale);
        const ff re = ff_mul(ff{v.x, v.y}, sc), im = ff_mul(ff{v.z, v.w}, sc);
        v = make_float4(re.h, re.l, im.h, im.l);
      }
      reinterpret_cast<float4*>(out_)[o] = v;
    } else {
      cd v = mkc(((double)rh + (double)rl) * scale, ((double)ih + (double)il) * scale);
      cd* d = reinterpret_cast<cd*>(out_) + o;
      *d = accumulate ? cadd(*d, v) : v;
    }
  }
}

template <bool IN_FF, bool OUT_FF>
static fmpb_status dft_axis(const char* name, const void* in, void* out, int O1, int O2, int64_t I, int64_t a1, int64_t a2, int64_t aj,
                            int64_t b1, int64_t b2, int64_t bf, int Pin, int Pout, int P, int sign, double scale,
                            bool accumulate, cudaStream_t st) {
  if (O1 > 65535 || O2 > 65535) {
    set_error("dft_axis: line grid %d x %d exceeds the launch limits", O1, O2);
    return FMPB_EINVAL;
  }
  if (OUT_FF && accumulate) {
    set_error("dft_axis: accumulation needs complex-double output");
    return FMPB_EINVAL;
  }
  // inner tile: up to 256 values (one per thread) so that long lines, such
  // as the operator's block columns, run in few CTAs that each amortise their
  // twiddle table; shrunk to the shared-memory budget and to fill the GPU
  // two-factor form when it saves at least a fifth of the products
  int P1 = 0;
  {
    const int64_t direct = (int64_t)Pout * Pin;
    int64_t best = direct;
    for (int a = 2; a * 2 <= P; ++a) {
      if (P % a) continue;
      const int b = P / a;
      const int64_t cost = (int64_t)a * Pin + P + (int64_t)Pout * b;
      if (cost < best) {
        best = cost;
        P1 = a;
      }
    }
    if (5 * best > 4 * direct) P1 = 0;
  }
  const int per_ti = Pin + (P1 > 0 ? P : 0);   // shared float4 values per inner index
  const size_t budget = 96 * 1024;
  int64_t TI = 256;
  while (TI > 1 && (size_t)(per_ti * TI + P) * sizeof(float4) > budget) TI /= 2;
  if ((size_t)(per_ti * TI + P) * sizeof(float4) > 200 * 1024) {
    set_error("dft_axis: axis length %d too large", P);
    return FMPB_EINVAL;
  }
  if (TI > I) TI = I;
  // enough CTAs to fill the 152 SMs several times over: shrink the inner
  // tile (down to 4 values, 64-byte segments) while the grid is small
  while (TI > 4 && ((I + TI - 1) / TI) * (int64_t)O1 * O2 < 4 * 152) TI /= 2;
  size_t smem = (size_t)(per_ti * TI + P) * sizeof(float4);
  FMPB_CUDA((smem_limit_once<k_dft_axis_ff<IN_FF, OUT_FF>>(200 * 1024)));
  dim3 grid((unsigned)((I + TI - 1) / TI), (unsigned)O2, (unsigned)O1);
  FMPB_LAUNCH(name, st, k_dft_axis_ff<IN_FF, OUT_FF><<<grid, 256, smem, st>>>(in, out, O2, I, a1, a2, aj, b1, b2, bf, Pin, Pout, P,
                                                                           sign, scale, accumulate ? 1 : 0, (int)TI, P1));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// One pass along an axis: the two-factor kernel of dft.cu wherever the
// length splits into factors of at most 16, else the direct float-float
// kernel above (a few long axes).
static fmpb_status axis_pass(const char* name, bool ff_arith, int in_fmt, int out_fmt, const void* in, void* out,
                             int O1, int O2, int64_t I, int64_t a1, int64_t a2, int64_t aj, int64_t b1, int64_t b2,
                             int64_t bf, int Pin, int Pout, int P, int sign, double scale, bool accumulate,
                             cudaStream_t st, int64_t row_b = 0, int row_kh = 0) {
  if (dft_supported(P))
    return dft_pass(name, ff_arith, in_fmt, out_fmt, in, out, O1, O2, I, a1, a2, aj, b1, b2, bf, Pin, Pout, P, sign,
                    scale, accumulate, st, row_b, row_kh);
  if (ff_arith) {
    if (in_fmt == DFT_CD && out_fmt == DFT_FF)
      return dft_axis<false, true>(name, in, out, O1, O2, I, a1, a2, aj, b1, b2, bf, Pin, Pout, P, sign, scale,
                                   accumulate, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_FF)
      return dft_axis<true, true>(name, in, out, O1, O2, I, a1, a2, aj, b1, b2, bf, Pin, Pout, P, sign, scale,
                                  accumulate, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_CD)
      return dft_axis<true, false>(name, in, out, O1, O2, I, a1, a2, aj, b1, b2, bf, Pin, Pout, P, sign, scale,
                                   accumulate, st);
  }
  set_error("%s: axis length %d needs the direct float-float pass", name, P);
  return FMPB_EINVAL;
}

bool circulant_f32_ok(const CircShape& s) {
  for (int a = 0; a < 3; ++a)
    if (s.P[a] > 1 && !dft_supported(s.P[a])) return false;
  return true;
}

// In-place forward DFT of a complex-double grid of F slots x `inner`
// values; the result is left in float-float format (the first pass converts).
fmpb_status grid_fft_inplace(const CircShape& s, int64_t inner, cd* grid, cudaStream_t st) {
  const int Px = s.P[0], Py = s.P[1], Pz = s.P[2];
  bool ff = false;
  if (Px > 1) {
    FMPB_TRY(axis_pass("dft_spectrum", true, DFT_CD, DFT_FF, grid, grid, 1, Pz * Py, inner, 0, (int64_t)Px * inner,
                       inner, 0, (int64_t)Px * inner, inner, Px, Px, Px, -1, 1.0, false, st));
    ff = true;
  }
  if (Py > 1) {
    FMPB_TRY(axis_pass("dft_spectrum", true, ff ? DFT_FF : DFT_CD, DFT_FF, grid, grid, Pz, Px, inner,
                       (int64_t)Py * Px * inner, inner, (int64_t)Px * inner, (int64_t)Py * Px * inner, inner,
                       (int64_t)Px * inner, Py, Py, Py, -1, 1.0, false, st));
    ff = true;
  }
  if (Pz > 1) {
    FMPB_TRY(axis_pass("dft_spectrum", true, ff ? DFT_FF : DFT_CD, DFT_FF, grid, grid, 1, Py * Px, inner, 0, inner,
                       (int64_t)Py * Px * inner, 0, inner, (int64_t)Py * Px * inner, Pz, Pz, Pz, -1, 1.0, false, st));
    ff = true;
  }
  if (!ff) FMPB_TRY(spectrum_to_ff(grid, (size_t)s.F * inner, st));
  return FMPB_OK;
}

// Y_f[r][b] = sum_b' Lambda_f[b][b'] X_f[r][b'] in float-float arithmetic.
// X_f, Y_f are float-float (float4); the spectrum is float-float (SPEC_FF, the
// operator's format) or complex double (split on the fly; the building-block
// API keeps its spectrum in FP64).  One warp per row, 4 independent 16-byte
// loads in flight per lane, X_f staged in shared memory for RC right-hand
// sides at a time.
template <int RC, bool SPEC_FF>
__global__ void __launch_bounds__(256) k_block_product_ff(const void* __restrict__ spec_, const float4* __restrict__ X,
                                                          float4* __restrict__ Y, int64_t B, int R, int r0,
                                                          int rows_per_cta) {
  extern __shared__ float4 xs4[];   // RC x B
  const int64_t f = blockIdx.y;
  const int64_t RB = (int64_t)R * B;
  const float4* Xf = X + f * RB + (int64_t)r0 * B;
  const int rc = min(RC, R - r0);
  for (int64_t e = threadIdx.x; e < (int64_t)rc * B; e += blockDim.x) xs4[e] = Xf[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int64_t bend = min(B, (int64_t)(blockIdx.x + 1) * rows_per_cta);
  for (int64_t b = (int64_t)blockIdx.x * rows_per_cta + warp; b < bend; b += nwarps) {
    float rh[RC], rl[RC], ih[RC], il[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) rh[r] = rl[r] = ih[r] = il[r] = 0.f;
    const int64_t row0 = (f * B + b) * B;
    auto load = [&](int64_t k) -> float4 {
      if (SPEC_FF) return __ldcs(reinterpret_cast<const float4*>(spec_) + row0 + k);
      return split_ff(reinterpret_cast<const cd*>(spec_)[row0 + k]);
    };
    int64_t bp = lane;
    for (; bp + 96 < B; bp += 128) {
      float4 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = load(bp + 32 * u);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int r = 0; r < RC; ++r)
          if (r < rc) ff_cmac(a[u], xs4[r * B + bp + 32 * u], rh[r], rl[r], ih[r], il[r]);
    }
    for (; bp < B; bp += 32) {
      const float4 a = load(bp);
#pragma unroll
      for (int r = 0; r < RC; ++r)
        if (r < rc) ff_cmac(a, xs4[r * B + bp], rh[r], rl[r], ih[r], il[r]);
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      ff_warp_sum(rh[r], rl[r]);
      ff_warp_sum(ih[r], il[r]);
      if (lane == 0 && r < rc) Y[f * RB + (int64_t)(r0 + r) * B + b] = ff_norm(rh[r], rl[r], ih[r], il[r]);
    }
  }
}

// In-place conversion of a complex-double array to float-float pairs.
__global__ void k_to_ff(cd* __restrict__ a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cd v = a[i];
    reinterpret_cast<float4*>(a)[i] = split_ff(v);
  }
}

// In-place conversion of float-float pairs back to complex double.
__global__ void k_from_ff(cd* __restrict__ a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(a)[i];
    a[i] = ff_to_cd(v);
  }
}

fmpb_status spectrum_to_ff(cd* spec, size_t n, cudaStream_t st) {
  FMPB_LAUNCH("to_ff", st, k_to_ff<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(spec, n));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

__global__ void k_vec_to_ff(const cd* __restrict__ x, float4* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = split_ff(x[i]);
}

__global__ void k_vec_to_f32(const cd* __restrict__ x, float2* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

fmpb_status vector_to_f32(const cd* x, float2* y, size_t n, cudaStream_t st) {
  FMPB_LAUNCH("to_f32", st, k_vec_to_f32<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(x, y, n));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status vector_to_ff(const cd* x, float4* y, size_t n, cudaStream_t st) {
  FMPB_LAUNCH("to_ff", st, k_vec_to_ff<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(x, y, n));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

static fmpb_status spectrum_from_ff(cd* spec, size_t n, cudaStream_t st) {
  FMPB_LAUNCH("from_ff", st, k_from_ff<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(spec, n));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// Y_f = Lambda_f X_f with Lambda_f in complex FP32 (mixed-precision operator):
// X_f (float-float) is rounded to FP32 in shared memory, products and sums
// are FP32, Y_f is written as float-float with a zero low part.  8-byte
// spectrum entries halve the bytes streamed per product.
// XT: float4 (float-float frequency values, output with a zero low part) or
// float2 (complex FP32 frequency values of FP32 DFT passes).
__device__ __forceinline__ float2 to_f32(float4 v) { return make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w)); }
__device__ __forceinline__ float2 to_f32(float2 v) { return v; }
template <typename XT>
__device__ __forceinline__ XT from_f32(float re, float im);
template <>
__device__ __forceinline__ float4 from_f32<float4>(float re, float im) {
  return make_float4(re, 0.f, im, 0.f);
}
template <>
__device__ __forceinline__ float2 from_f32<float2>(float re, float im) {
  return make_float2(re, im);
}

template <int RC, typename XT>
__global__ void __launch_bounds__(256) k_block_product_f32(const float2* __restrict__ spec, const XT* __restrict__ X,
                                                           XT* __restrict__ Y, int64_t B, int R, int r0,
                                                           int rows_per_cta) {
  extern __shared__ float2 xs2[];   // RC x B
  const int64_t f = blockIdx.y;
  const int64_t RB = (int64_t)R * B;
  const XT* Xf = X + f * RB + (int64_t)r0 * B;
  const int rc = min(RC, R - r0);
  for (int64_t e = threadIdx.x; e < (int64_t)rc * B; e += blockDim.x) xs2[e] = to_f32(Xf[e]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int64_t bend = min(B, (int64_t)(blockIdx.x + 1) * rows_per_cta);
  for (int64_t b = (int64_t)blockIdx.x * rows_per_cta + warp; b < bend; b += nwarps) {
    float re[RC], im[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) re[r] = im[r] = 0.f;
    const float2* row = spec + (f * B + b) * B;
    int64_t bp = lane;
    for (; bp + 224 < B; bp += 256) {
      float2 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcs(row + bp + 32 * u);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int r = 0; r < RC; ++r)
          if (r < rc) {
            const float2 x = xs2[r * B + bp + 32 * u];
            re[r] = fmaf(a[u].x, x.x, fmaf(-a[u].y, x.y, re[r]));
            im[r] = fmaf(a[u].x, x.y, fmaf(a[u].y, x.x, im[r]));
          }
    }
    for (; bp < B; bp += 32) {
      const float2 a = __ldcs(row + bp);
#pragma unroll
      for (int r = 0; r < RC; ++r)
        if (r < rc) {
          const float2 x = xs2[r * B + bp];
          re[r] = fmaf(a.x, x.x, fmaf(-a.y, x.y, re[r]));
          im[r] = fmaf(a.x, x.y, fmaf(a.y, x.x, im[r]));
        }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      for (int o = 16; o > 0; o >>= 1) {
        re[r] += __shfl_xor_sync(0xffffffffu, re[r], o);
        im[r] += __shfl_xor_sync(0xffffffffu, im[r], o);
      }
      if (lane == 0 && r < rc) Y[f * RB + (int64_t)(r0 + r) * B + b] = from_f32<XT>(re[r], im[r]);
    }
  }
}

template <int RC, typename XT>
static fmpb_status launch_block_product_f32(const float2* spec, const XT* X, XT* Y, int64_t F, int64_t B,
                                            int R, cudaStream_t st) {
  const int threads = 256, rows = 32;
  const size_t smem = (size_t)RC * B * sizeof(float2);
  FMPB_CUDA((smem_limit_once<k_block_product_f32<RC, XT>>(200 * 1024)));
  dim3 grid((unsigned)((B + rows - 1) / rows), (unsigned)F);
  for (int r0 = 0; r0 < R; r0 += RC) {
    FMPB_LAUNCH("block_product_f32", st, k_block_product_f32<RC, XT><<<grid, threads, smem, st>>>(spec, X, Y, B, R, r0, rows));
    FMPB_CUDA(cudaGetLastError());
  }
  return FMPB_OK;
}

// float-float spectrum (16 bytes per entry) -> complex FP32 (8 bytes)
__global__ void k_ff_to_f32(const float4* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[i] = make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
  }
}

fmpb_status spectrum_ff_to_f32(const cd* in, void* out, size_t n, cudaStream_t st) {
  FMPB_LAUNCH("to_f32", st, k_ff_to_f32<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(reinterpret_cast<const float4*>(in), reinterpret_cast<float2*>(out), n));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

template <int RC, bool SPEC_FF>
static fmpb_status launch_block_product(const void* spec, const float4* X, float4* Y, int64_t F, int64_t B, int R,
                                        cudaStream_t st) {
  const int threads = 256, rows = 32;
  const size_t smem = (size_t)RC * B * sizeof(float4);
  FMPB_CUDA((smem_limit_once<k_block_product_ff<RC, SPEC_FF>>(200 * 1024)));
  dim3 grid((unsigned)((B + rows - 1) / rows), (unsigned)F);
  for (int r0 = 0; r0 < R; r0 += RC) {
    FMPB_LAUNCH("block_product", st, k_block_product_ff<RC, SPEC_FF><<<grid, threads, smem, st>>>(spec, X, Y, B, R, r0, rows));
    FMPB_CUDA(cudaGetLastError());
  }
  return FMPB_OK;
}

// Many right-hand sides: Y_f[r][b] = sum_k X_f[r][k] Lambda_f[b][k] as a
// tiled GEMM per frequency.  A CTA owns 32 rows b x 32 right-hand sides r and
// walks k in slices of 16 through shared memory; each thread accumulates 2 x 2
// outputs.  The r-tile index is the fastest grid dimension, so the CTAs that
// share a spectrum tile run together and reuse it from L2.  FF: float-float
// spectrum and arithmetic; otherwise complex FP32 spectrum and FP32 FMAs.
constexpr int BPT_B = 32, BPT_R = 32, BPT_K = 16;
__device__ __forceinline__ float4 to_ff4(float4 v) { return v; }
__device__ __forceinline__ float4 to_ff4(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }
template <bool FF, typename XT>
__global__ void __launch_bounds__(256) k_block_product_tiled(const void* __restrict__ spec_,
                                                             const XT* __restrict__ X, XT* __restrict__ Y,
                                                             int64_t B, int R) {
  __shared__ float4 Ls[BPT_B][BPT_K + 1];
  __shared__ float4 Xs[BPT_K][BPT_R + 1];
  const int64_t f = blockIdx.y;
  const int r0 = blockIdx.x * BPT_R;
  const int64_t b0 = (int64_t)blockIdx.z * BPT_B;
  const int64_t RB = (int64_t)R * B;
  const XT* Xf = X + f * RB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float rh[2][2], rl[2][2], ih[2][2], il[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) rh[a][b] = rl[a][b] = ih[a][b] = il[a][b] = 0.f;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k0 = 0; k0 < B; k0 += BPT_K) {
    for (int e = threadIdx.x; e < BPT_B * BPT_K; e += blockDim.x) {
      const int bb = e / BPT_K, kk = e - bb * BPT_K;
      const int64_t b = b0 + bb, k = k0 + kk;
      float4 v = zero;
      if (b < B && k < B) {
        const int64_t idx = (f * B + b) * B + k;
        if (FF) {
          v = __ldcs(reinterpret_cast<const float4*>(spec_) + idx);
        } else {
          const float2 s = __ldcs(reinterpret_cast<const float2*>(spec_) + idx);
          v = make_float4(s.x, 0.f, s.y, 0.f);
        }
      }
      Ls[bb][kk] = v;
    }
    for (int e = threadIdx.x; e < BPT_R * BPT_K; e += blockDim.x) {
      const int rr = e / BPT_K, kk = e - rr * BPT_K;
      const int r = r0 + rr;
      const int64_t k = k0 + kk;
      Xs[kk][rr] = (r < R && k < B) ? to_ff4(Xf[(int64_t)r * B + k]) : zero;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BPT_K; ++kk) {
      const float4 l0 = Ls[ty][kk], l1 = Ls[ty + 16][kk];
      const float4 x0 = Xs[kk][tx], x1 = Xs[kk][tx + 16];
      if (FF) {
        ff_cmac(l0, x0, rh[0][0], rl[0][0], ih[0][0], il[0][0]);
        ff_cmac(l0, x1, rh[0][1], rl[0][1], ih[0][1], il[0][1]);
        ff_cmac(l1, x0, rh[1][0], rl[1][0], ih[1][0], il[1][0]);
        ff_cmac(l1, x1, rh[1][1], rl[1][1], ih[1][1], il[1][1]);
      } else {
        const float4* ls[2] = {&l0, &l1};
        const float4* xs[2] = {&x0, &x1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const float lr = ls[a]->x, li = ls[a]->z;
            const float xr = xs[b]->x + xs[b]->y, xi = xs[b]->z + xs[b]->w;
            rh[a][b] = fmaf(lr, xr, fmaf(-li, xi, rh[a][b]));
            ih[a][b] = fmaf(lr, xi, fmaf(li, xr, ih[a][b]));
          }
      }
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int64_t row = b0 + ty + 16 * a;
      const int r = r0 + tx + 16 * b;
      if (row < B && r < R) {
        if constexpr (FF)
          Y[f * RB + (int64_t)r * B + row] = ff_norm(rh[a][b], rl[a][b], ih[a][b], il[a][b]);
        else
          Y[f * RB + (int64_t)r * B + row] = from_f32<XT>(rh[a][b], ih[a][b]);
      }
    }
}

template <bool FF, typename XT>
static fmpb_status launch_block_product_tiled(const void* spec, const XT* X, XT* Y, int64_t F, int64_t B,
                                              int R, cudaStream_t st) {
  const int64_t btiles = (B + BPT_B - 1) / BPT_B;
  if (btiles > 65535) {
    set_error("block_product: block size %lld too large", (long long)B);
    return FMPB_EINVAL;
  }
  dim3 grid((unsigned)((R + BPT_R - 1) / BPT_R), (unsigned)F, (unsigned)btiles);
  FMPB_LAUNCH(FF ? "block_product_tiled" : "block_product_tiled_f32", st, k_block_product_tiled<FF, XT><<<grid, 256, 0, st>>>(spec, X, Y, B, R));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// X, Y: the frequency-domain values [f][r][b], float-float (float4) or, with
// f32_io, complex FP32 (float2; FP32 and BF16 spectra only).
static fmpb_status block_product(const void* spec, int spec_format, const void* Xv, void* Yv, int64_t F,
                                 int64_t B, int R, cudaStream_t st, void* tc_rows, unsigned* tc_err,
                                 bool f32_io = false, const void* const* spec_batch = nullptr, int n_ops = 1,
                                 const int* batch_blk = nullptr, int n_blocks = 0, bool rows_ready = false) {
  if (spec_batch) {
    const int nb = n_blocks > 0 ? n_blocks : n_ops;
    if (spec_format != SPEC_BF16 || n_ops < 1 || nb < n_ops || R % nb || !tc_rows || !tc_err) {
      set_error("block_product: a batch of operators takes BF16 spectra and R a multiple of the operator count");
      return FMPB_EINVAL;
    }
    if (n_ops > TC_MAX_BATCH) {
      set_error("block_product: %d operators in a batch (1..%d)", n_ops, TC_MAX_BATCH);
      return FMPB_EINVAL;
    }
    const __nv_bfloat16* A[TC_MAX_BATCH];
    for (int o = 0; o < n_ops; ++o) A[o] = reinterpret_cast<const __nv_bfloat16*>(spec_batch[o]);
    __nv_bfloat16* rows = reinterpret_cast<__nv_bfloat16*>(tc_rows);
    if (rows_ready) {
    } else if (f32_io) {
      FMPB_TRY(tc_rows_from_f32(reinterpret_cast<const float2*>(Xv), F * R, B, rows, st));
    } else {
      FMPB_TRY(tc_rows_from_ff(reinterpret_cast<const float4*>(Xv), F * R, B, rows, st));
    }
    return tc_freq_gemm_batch(A, n_ops, F, B, R / nb, rows, Yv, tc_err, st, f32_io, batch_blk, nb);
  }
  if (F > 65535) {
    set_error("block_product: %lld frequencies exceed the launch limit", (long long)F);
    return FMPB_EINVAL;
  }
  if (f32_io) {
    if (spec_format != SPEC_F32 && spec_format != SPEC_BF16) {
      set_error("block_product: FP32 frequency values take an FP32 or BF16 spectrum");
      return FMPB_EINVAL;
    }
    const float2* X2 = reinterpret_cast<const float2*>(Xv);
    float2* Y2 = reinterpret_cast<float2*>(Yv);
    if (spec_format == SPEC_BF16) {
      if (!tc_rows || !tc_err) {
        set_error("block_product: BF16 spectrum without tensor-core scratch");
        return FMPB_EINVAL;
      }
      __nv_bfloat16* rows = reinterpret_cast<__nv_bfloat16*>(tc_rows);
      if (!rows_ready) FMPB_TRY(tc_rows_from_f32(X2, F * R, B, rows, st));
      return tc_freq_gemm(reinterpret_cast<const __nv_bfloat16*>(spec), F, B, R, rows, Y2, tc_err, st, true);
    }
    if (R >= 8) return launch_block_product_tiled<false, float2>(spec, X2, Y2, F, B, R, st);
    const int RC2 = R >= 4 ? 4 : (R >= 2 ? 2 : 1);
    if ((size_t)RC2 * B * sizeof(float2) > 200 * 1024) {
      set_error("block_product: block size %lld too large", (long long)B);
      return FMPB_EINVAL;
    }
    const float2* sp = reinterpret_cast<const float2*>(spec);
    if (RC2 == 4) return launch_block_product_f32<4, float2>(sp, X2, Y2, F, B, R, st);
    if (RC2 == 2) return launch_block_product_f32<2, float2>(sp, X2, Y2, F, B, R, st);
    return launch_block_product_f32<1, float2>(sp, X2, Y2, F, B, R, st);
  }
  const float4* X = reinterpret_cast<const float4*>(Xv);
  float4* Y = reinterpret_cast<float4*>(Yv);
  // BF16 spectrum: every frequency's product on the tensor cores
  if (spec_format == SPEC_BF16) {
    if (!tc_rows || !tc_err) {
      set_error("block_product: BF16 spectrum without tensor-core scratch");
      return FMPB_EINVAL;
    }
    __nv_bfloat16* rows = reinterpret_cast<__nv_bfloat16*>(tc_rows);
    FMPB_TRY(tc_rows_from_ff(X, F * R, B, rows, st));
    return tc_freq_gemm(reinterpret_cast<const __nv_bfloat16*>(spec), F, B, R, rows, Y, tc_err, st);
  }
  // many right-hand sides: one tiled pass over the spectrum
  if (R >= 8 && spec_format == SPEC_FF) return launch_block_product_tiled<true, float4>(spec, X, Y, F, B, R, st);
  if (R >= 8 && spec_format == SPEC_F32) return launch_block_product_tiled<false, float4>(spec, X, Y, F, B, R, st);
  const int RC = R >= 4 ? 4 : (R >= 2 ? 2 : 1);
  if ((size_t)RC * B * sizeof(float4) > 200 * 1024) {
    set_error("block_product: block size %lld too large", (long long)B);
    return FMPB_EINVAL;
  }
  if (spec_format == SPEC_F32) {
    const float2* sp = reinterpret_cast<const float2*>(spec);
    if (RC == 4) return launch_block_product_f32<4, float4>(sp, X, Y, F, B, R, st);
    if (RC == 2) return launch_block_product_f32<2, float4>(sp, X, Y, F, B, R, st);
    return launch_block_product_f32<1, float4>(sp, X, Y, F, B, R, st);
  }
  if (spec_format == SPEC_FF) {
    if (RC == 4) return launch_block_product<4, true>(spec, X, Y, F, B, R, st);
    if (RC == 2) return launch_block_product<2, true>(spec, X, Y, F, B, R, st);
    return launch_block_product<1, true>(spec, X, Y, F, B, R, st);
  }
  if (RC == 4) return launch_block_product<4, false>(spec, X, Y, F, B, R, st);
  if (RC == 2) return launch_block_product<2, false>(spec, X, Y, F, B, R, st);
  return launch_block_product<1, false>(spec, X, Y, F, B, R, st);
}

size_t circulant_scratch_elems(const CircShape& s, int64_t B, int R) { return 2 * (size_t)s.F * R * B; }

fmpb_status circulant_apply(const CircShape& s, int64_t B, const cd* spec, int R, const cd* x, cd* y,
                            bool accumulate, cd* scratch, cudaStream_t st, int spec_format, void* tc_rows,
                            unsigned* tc_err, bool ff_io, bool f32_passes, const void* const* spec_batch,
                            int n_ops, const int* batch_blk, int n_blocks, void* y_rows) {
  const int Mx = s.M[0], My = s.M[1], Mz = s.M[2];
  const int Px = s.P[0], Py = s.P[1], Pz = s.P[2];
  const int64_t RB = (int64_t)R * B;
  const int64_t Nc = s.ncells;
  if (f32_passes && (ff_io || (spec_format != SPEC_F32 && spec_format != SPEC_BF16) || !circulant_f32_ok(s))) {
    set_error("circulant_apply: FP32 passes take an FP32 or BF16 spectrum, complex-double vectors and axis lengths "
              "that split into factors of at most 16");
    return FMPB_EINVAL;
  }
  // two buffers of frequency-domain values: float-float (16 bytes per value,
  // like complex double) or complex FP32 (8 bytes); an axis with a single
  // cell (P = 1) leaves the layout unchanged and is skipped
  const bool ffa = !f32_passes;
  const size_t vb = ffa ? sizeof(float4) : sizeof(float2);
  char* sb = reinterpret_cast<char*>(scratch);
  void* buf[2] = {sb, sb + (size_t)s.F * RB * vb};
  const int mid = ffa ? DFT_FF : DFT_F32;
  const int io = ff_io ? DFT_FF : DFT_CD;
  // FP32 passes ahead of tensor-core products: the last forward pass writes
  // the BF16 rows of the products itself (no FP32 frequency values and no
  // conversion pass); row f R + r holds the B values of (f, r)
  const int last = Pz > 1 ? 2 : (Py > 1 ? 1 : 0);
  const int lastP = s.P[last], lastM = s.M[last];
  const bool rows = !ffa && spec_format == SPEC_BF16 && tc_rows && dft_supported(lastP) &&
                    dft_rows_ok(lastP, lastM);
  const int row_kh = (int)(tc_depth(B) / 2);
  auto fwd_out = [&](int axis, int cur_fmt, void* dst) -> std::pair<int, void*> {
    return rows && axis == last ? std::make_pair((int)DFT_BF16R, tc_rows) : std::make_pair(cur_fmt, dst);
  };
  int cur = 0;
  // forward x: x[r][cz][cy][cx][b] -> [cz][cy][fx][r][b]
  {
    const auto o = fwd_out(0, mid, buf[cur]);
    FMPB_TRY(axis_pass("dft_fwd_x", ffa, io, o.first, x, o.second, R, Mz * My, B, Nc * B, (int64_t)Mx * B, B, B,
                       (int64_t)Px * RB, RB, Mx, Px, Px, -1, 1.0, false, st, B, row_kh));
  }
  // forward y: [cz][cy][fx][rb] -> [cz][fy][fx][rb]
  if (Py > 1) {
    const auto o = fwd_out(1, mid, buf[1 - cur]);
    FMPB_TRY(axis_pass("dft_fwd_y", ffa, mid, o.first, buf[cur], o.second, Mz, Px, RB, (int64_t)My * Px * RB, RB,
                       (int64_t)Px * RB, (int64_t)Py * Px * RB, RB, (int64_t)Px * RB, My, Py, Py, -1, 1.0, false, st,
                       B, row_kh));
    cur = 1 - cur;
  }
  // forward z: [cz][fy fx][rb] -> [fz][fy fx][rb]
  if (Pz > 1) {
    const auto o = fwd_out(2, mid, buf[1 - cur]);
    FMPB_TRY(axis_pass("dft_fwd_z", ffa, mid, o.first, buf[cur], o.second, 1, Py * Px, RB, 0, RB,
                       (int64_t)Py * Px * RB, 0, RB, (int64_t)Py * Px * RB, Mz, Pz, Pz, -1, 1.0, false, st, B,
                       row_kh));
    cur = 1 - cur;
  }
  // per-frequency block products: [f][r][b] -> [f][r][b]
  FMPB_TRY(block_product(spec, spec_format, buf[cur], buf[1 - cur], s.F, B, R, st, tc_rows, tc_err, !ffa,
                         spec_batch, n_ops, batch_blk, n_blocks, rows));
  cur = 1 - cur;
  // inverse z: [fz][fy fx][rb] -> [cz][fy fx][rb], cz < Mz
  if (Pz > 1) {
    FMPB_TRY(axis_pass("dft_inv_z", ffa, mid, mid, buf[cur], buf[1 - cur], 1, Py * Px, RB, 0, RB,
                       (int64_t)Py * Px * RB, 0, RB, (int64_t)Py * Px * RB, Pz, Mz, Pz, +1, 1.0, false, st));
    cur = 1 - cur;
  }
  // inverse y: [cz][fy][fx][rb] -> [cz][cy][fx][rb], cy < My
  if (Py > 1) {
    FMPB_TRY(axis_pass("dft_inv_y", ffa, mid, mid, buf[cur], buf[1 - cur], Mz, Px, RB, (int64_t)Py * Px * RB, RB,
                       (int64_t)Px * RB, (int64_t)My * Px * RB, RB, (int64_t)Px * RB, Py, My, Py, +1, 1.0, false, st));
    cur = 1 - cur;
  }
  // inverse x with crop and 1/F: [cz][cy][fx][r][b] -> y[r][cz][cy][cx][b]
  // (or straight into the BF16 rows of a tensor-core product, row r Nc + c)
  if (y_rows) {
    if (ffa || accumulate || !dft_supported(Px) || !dft_rows_ok(Px, Px)) {
      set_error("circulant_apply: BF16 result rows take FP32 passes without accumulation");
      return FMPB_EINVAL;
    }
    FMPB_TRY(axis_pass("dft_inv_x", ffa, mid, DFT_BF16R, buf[cur], y_rows, R, Mz * My, B, B, (int64_t)Px * RB, RB,
                       Nc * B, (int64_t)Mx * B, B, Px, Mx, Px, +1, 1.0 / (double)s.F, false, st, B, row_kh));
    return FMPB_OK;
  }
  FMPB_TRY(axis_pass("dft_inv_x", ffa, mid, io, buf[cur], y, R, Mz * My, B, B, (int64_t)Px * RB, RB, Nc * B,
                     (int64_t)Mx * B, B, Px, Mx, Px, +1, 1.0 / (double)s.F, accumulate, st));
  return FMPB_OK;
}

// out[r][c][i] = in[r][P c][i]: the cells of every right-hand side reversed
// along lattice axis h (the permutation P of the block Hankel image part of a
// half-space operator, Sec. 2.4).  in and out do not overlap.
template <typename T>
__global__ void k_reverse_cells(const T* __restrict__ in, T* __restrict__ out, int64_t total, int n, int Mx, int My,
                                int Mz, int h) {
  const int64_t Nc = (int64_t)Mx * My * Mz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const int64_t rc = idx / n;
    const int c = (int)(rc % Nc);
    const int64_t r = rc / Nc;
    int cx = c % Mx, cy = (c / Mx) % My, cz = c / (Mx * My);
    if (h == 0) cx = Mx - 1 - cx;
    if (h == 1) cy = My - 1 - cy;
    if (h == 2) cz = Mz - 1 - cz;
    out[idx] = in[(r * Nc + ((int64_t)cz * My + cy) * Mx + cx) * n + i];
  }
}

fmpb_status reverse_cells(const void* in, void* out, size_t elem_bytes, int R, const int M[3], int n, int h,
                          cudaStream_t st) {
  if (h < 0 || h > 2 || (elem_bytes != 8 && elem_bytes != 16)) {
    set_error("reverse_cells: bad axis or element size");
    return FMPB_EINVAL;
  }
  const int64_t total = (int64_t)R * M[0] * M[1] * M[2] * n;
  const unsigned grid = (unsigned)std::min<int64_t>(grid_for(total, 256), 152 * 32);
  if (elem_bytes == 16)
    FMPB_LAUNCH("reverse_cells", st, k_reverse_cells<float4><<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(in), reinterpret_cast<float4*>(out), total, n, M[0], M[1], M[2], h));
  else
    FMPB_LAUNCH("reverse_cells", st, k_reverse_cells<float2><<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), total, n, M[0], M[1], M[2], h));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

__global__ void k_scale_cd(cd* __restrict__ a, size_t n, cd s) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = cmul(s, a[i]);
}

fmpb_status scale_inplace(cd* a, size_t n, cd s, cudaStream_t st) {
  FMPB_LAUNCH("scale", st, k_scale_cd<<<std::min<size_t>(grid_for(n, 256), 152 * 32), 256, 0, st>>>(a, n, s));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// Scatter blocks given in offset order (delta_x fastest, 1-M..M-1) into the
// zeroed padded grid.
__global__ void k_scatter_offsets(const cd* __restrict__ blocks, cd* __restrict__ grid, int64_t BB,
                                  const int64_t* __restrict__ slot, int n_off) {
  const size_t total = (size_t)BB * n_off;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx / BB);
    const int64_t e = (int64_t)(idx - (size_t)o * BB);
    grid[(size_t)slot[o] * BB + e] = blocks[idx];
  }
}

fmpb_status circulant_spectrum_from_blocks(const CircShape& s, int64_t B, const cd* blocks, cd* spec,
                                           cudaStream_t st) {
  std::vector<int64_t> slots;
  for (int dz = 1 - s.M[2]; dz < s.M[2]; ++dz)
    for (int dy = 1 - s.M[1]; dy < s.M[1]; ++dy)
      for (int dx = 1 - s.M[0]; dx < s.M[0]; ++dx) slots.push_back(offset_slot(s, dx, dy, dz));
  const int n_off = (int)slots.size();
  int64_t* dslot = nullptr;
  FMPB_CUDA(cudaMallocAsync(&dslot, sizeof(int64_t) * n_off, st));
  FMPB_CUDA(cudaMemcpyAsync(dslot, slots.data(), sizeof(int64_t) * n_off, cudaMemcpyHostToDevice, st));
  FMPB_CUDA(cudaMemsetAsync(spec, 0, sizeof(cd) * (size_t)s.F * B * B, st));
  const size_t total = (size_t)B * B * n_off;
  FMPB_LAUNCH("scatter_offsets", st, k_scatter_offsets<<<std::min<size_t>(grid_for(total, 256), 152 * 32), 256, 0, st>>>(blocks, spec, B * B, dslot,
                                                                                       n_off));
  FMPB_CUDA(cudaGetLastError());
  FMPB_TRY(grid_fft_inplace(s, B * B, spec, st));
  // the building-block API returns the spectrum in complex double
  FMPB_TRY(spectrum_from_ff(spec, (size_t)s.F * B * B, st));
  FMPB_CUDA(cudaFreeAsync(dslot, st));
  return FMPB_OK;
}

}  // namespace fmpb

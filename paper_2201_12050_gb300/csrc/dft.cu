// Pruned DFT passes of the circulant engine (Sec. 2.4, Eqs. (diagonalized),
// (modifiedFourierTransform1), (modifiedFourierTransform2)): along one axis
// of the padded cell grid, for every line (o1, o2) and inner index i,
//   out[o1 b1 + o2 b2 + f bf + i] (+)= scale sum_{j < Pin} in[o1 a1 + o2 a2 + j aj + i] w^{f j},
// w = exp(sign 2 pi i / P), f < Pout.  Pin < P for the forward transform of
// the zero-padded grid (the incomplete Fourier matrix), Pout < P for the
// cropped inverse.
//
// Algorithm: the two-factor (Cooley-Tukey) split P = P1 P2, n = P2 n1 + n2,
// f = k1 + P1 k2:
//   stage A, per n2 < P2: Y[n2][k1] = w^{n2 k1} sum_{n1} in[P2 n1 + n2] w^{P2 n1 k1}   (k1 < P1)
//   stage B, per k1 < P1: out[k1 + P1 k2] = sum_{n2} Y[n2][k1] w^{P1 n2 k2}             (k2 < P2)
// with P1, P2 <= 16 chosen to minimise the complex multiply-adds (P2 = 1 is
// the direct sum).  Only the non-zero inputs are read and only the kept
// outputs are formed.  Two more forms need no shared-memory exchange: the
// direct sum (k_dft_direct, a thread's inputs all in flight at once) and,
// for FP32 lines of 8, 16 or 32, a radix-2 FFT in registers (k_dft_fft2).
// A pass runs the model's choice or, for a new line shape, the fastest of
// the forms it admits, timed once on its first call (the autotuner below).
//
// Layout on the GB300: a warp owns 32 consecutive inner indices (the
// contiguous dimension of every pass), so each of its loads and stores is
// one 256-byte (FP32) or 512-byte (float-float) coalesced transaction.  A
// stage-A item (n2, 32 inner indices) holds its up to 16 inputs in
// registers and forms the short DFT there; the P1 x P2 intermediate values
// go through shared memory to the stage-B items (k1, 32 inner indices),
// which again work from registers and store straight to global memory.
// Twiddles sit in shared memory and every lane of a warp reads the same one
// (a broadcast).  CTAs are persistent over tiles of (line, 32 nsub inner
// indices), so the twiddle tables are built once per CTA.
//
// Arithmetic: float-float (48-bit significands on the FP32 pipe, the FP64
// operators) or plain FP32 (8 bytes per value: the FP32, BF16 and
// mixed-precision inner operators, whose products carry 1e-5 or less
// accuracy anyway).  In place (in == out with equal strides, Pin = Pout = P)
// is allowed: every input of a tile is read before any output of it is
// written.
#include <cuda_bf16.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "internal.cuh"
#include "profile.cuh"

namespace fmpb {

namespace {

constexpr int DFT_R = 16;          // longest factor held in registers
constexpr int DFT_THREADS = 256;
constexpr int DFT_WAVES = 8;       // grid of a pass: at most this many waves of resident CTAs

template <bool FF>
using DVal = typename std::conditional<FF, float4, float2>::type;

template <bool FF>
__device__ __forceinline__ DVal<FF> dzero();
template <>
__device__ __forceinline__ float4 dzero<true>() {
  return make_float4(0.f, 0.f, 0.f, 0.f);
}
template <>
__device__ __forceinline__ float2 dzero<false>() {
  return make_float2(0.f, 0.f);
}

// w^m = exp(sign 2 pi i m / P) from an FP64 sincospi of the exact fraction m / P
template <bool FF>
__device__ __forceinline__ DVal<FF> twiddle(int m, int P, int sign) {
  double s, c;
  sincospi(2.0 * m / P, &s, &c);
  if constexpr (FF)
    return split_ff(mkc(c, sign * s));
  else
    return make_float2((float)c, (float)(sign * s));
}

template <bool FF, int FMT>
__device__ __forceinline__ DVal<FF> dload(const void* p, int64_t idx) {
  if constexpr (FMT == DFT_CD) {
    const cd v = reinterpret_cast<const cd*>(p)[idx];
    if constexpr (FF)
      return split_ff(v);
    else
      return make_float2((float)v.x, (float)v.y);
  } else if constexpr (FMT == DFT_FF) {
    const float4 v = reinterpret_cast<const float4*>(p)[idx];
    if constexpr (FF)
      return v;
    else
      return make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
  } else {
    const float2 v = reinterpret_cast<const float2*>(p)[idx];
    if constexpr (FF)
      return make_float4(v.x, 0.f, v.y, 0.f);
    else
      return v;
  }
}

template <bool FF, int FMT>
__device__ __forceinline__ void dstore(void* p, int64_t idx, DVal<FF> v, double scale, int accumulate) {
  if constexpr (FMT == DFT_CD) {
    cd d;
    if constexpr (FF)
      d = mkc(((double)v.x + (double)v.y) * scale, ((double)v.z + (double)v.w) * scale);
    else
      d = mkc((double)v.x * scale, (double)v.y * scale);
    cd* o = reinterpret_cast<cd*>(p) + idx;
    *o = accumulate ? cadd(*o, d) : d;
  } else if constexpr (FMT == DFT_FF) {
    static_assert(FF, "float-float output takes float-float arithmetic");
    if (scale != 1.0) {
      const ff sc = ff_from_d(scale);
      const ff re = ff_mul(ff{v.x, v.y}, sc), im = ff_mul(ff{v.z, v.w}, sc);
      v = make_float4(re.h, re.l, im.h, im.l);
    }
    reinterpret_cast<float4*>(p)[idx] = v;
  } else {
    static_assert(!FF, "FP32 output takes FP32 arithmetic");
    const float s = (float)scale;
    reinterpret_cast<float2*>(p)[idx] = make_float2(v.x * s, v.y * s);
  }
}

// sum_{n < nin} x[n] T[(n k) mod m], the register-resident short DFT
template <bool FF>
__device__ __forceinline__ DVal<FF> short_dft(const DVal<FF> (&x)[DFT_R], const DVal<FF>* __restrict__ T, int nin,
                                              int k, int m) {
  int idx = 0;
  if constexpr (FF) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll
    for (int n = 0; n < DFT_R; ++n)
      if (n < nin) {
        ff_cmac(T[idx], x[n], rh, rl, ih, il);
        idx += k;
        if (idx >= m) idx -= m;
      }
    return ff_norm(rh, rl, ih, il);
  } else {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int n = 0; n < DFT_R; ++n)
      if (n < nin) {
        const float2 t = T[idx];
        re = fmaf(t.x, x[n].x, fmaf(-t.y, x[n].y, re));
        im = fmaf(t.x, x[n].y, fmaf(t.y, x[n].x, im));
        idx += k;
        if (idx >= m) idx -= m;
      }
    return make_float2(re, im);
  }
}

template <bool FF>
__device__ __forceinline__ DVal<FF> dmul(DVal<FF> a, DVal<FF> w) {
  if constexpr (FF) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    ff_cmac(w, a, rh, rl, ih, il);
    return ff_norm(rh, rl, ih, il);
  } else {
    return make_float2(fmaf(w.x, a.x, -w.y * a.y), fmaf(w.x, a.y, w.y * a.x));
  }
}

struct DftArgs {
  const void* in;
  void* out;
  int64_t I, a1, a2, aj, b1, b2, bf;
  int O1, O2, Pin, Pout, P, P1, P2, nsub, sign, accumulate;
  double scale;
  int64_t tiles_i, tiles;
  // DFT_BF16R output: values per row, pairs per row, and the output strides
  // b1, b2, bf in rows (multiples of row_b)
  int64_t row_b, b1r, b2r, bfr;
  int row_kh;
};

// Store of value f of an item whose inner index i sits in row `rowbase`
// (plus f bfr) at pair `col` of the BF16 rows.
__device__ __forceinline__ void store_bf16r(const DftArgs& a, int64_t rowbase, int64_t col, int f, float2 v) {
  const float sc = (float)a.scale;
  __nv_bfloat162 p;
  p.x = __float2bfloat16_rn(v.x * sc);
  p.y = __float2bfloat16_rn(v.y * sc);
  reinterpret_cast<__nv_bfloat162*>(a.out)[(rowbase + (int64_t)f * a.bfr) * a.row_kh + col] = p;
}

// Storage type of the input format (what the copies move into shared memory).
template <int FMT>
struct DIn;
template <>
struct DIn<DFT_CD> {
  typedef double2 T;
};
template <>
struct DIn<DFT_FF> {
  typedef float4 T;
};
template <>
struct DIn<DFT_F32> {
  typedef float2 T;
};

template <int FMT, bool FF>
__device__ __forceinline__ DVal<FF> from_stored(typename DIn<FMT>::T v) {
  if constexpr (FMT == DFT_CD) {
    if constexpr (FF)
      return split_ff(v);
    else
      return make_float2((float)v.x, (float)v.y);
  } else if constexpr (FMT == DFT_FF) {
    if constexpr (FF)
      return v;
    else
      return make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
  } else {
    if constexpr (FF)
      return make_float4(v.x, 0.f, v.y, 0.f);
    else
      return v;
  }
}

// Asynchronous global -> shared copy of one 8- or 16-byte value; src_bytes
// 0 fills the destination with zeros (the pruned inputs past the grid).
template <int BYTES>
__device__ __forceinline__ void cp_async_val(uint32_t dst, const void* src, int src_bytes) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared memory of a CTA: twiddles (P + P1 + P2 values), the intermediate
// values Y (nsub x P x 32, two-factor plans only) and two input stages of
// Pin x 32 nsub stored values each (the next tile's copies overlap the
// current tile's arithmetic).
template <bool FF, int IN, int OUT>
__global__ void __launch_bounds__(DFT_THREADS, 2) k_dft(const DftArgs a) {
  using V = DVal<FF>;
  using S = typename DIn<IN>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  V* tw = reinterpret_cast<V*>(dsm);   // w^m, m < P
  V* t1 = tw + a.P;                    // w^{P2 m}, m < P1
  V* t2 = t1 + a.P1;                   // w^{P1 m}, m < P2
  V* Y = t2 + a.P2;                    // nsub x P x 32 intermediate values
  const int64_t TI = 32 * (int64_t)a.nsub;
  const int64_t ybytes = (a.P2 > 1 ? (int64_t)a.nsub * a.P * 32 : 0) * (int64_t)sizeof(V);
  const int64_t off = (((int64_t)(a.P + a.P1 + a.P2) * (int64_t)sizeof(V) + ybytes) + 15) / 16 * 16;
  S* stage = reinterpret_cast<S*>(dsm + off);   // [2][Pin][TI]
  const int64_t per_stage = (int64_t)a.Pin * TI;
  for (int m = threadIdx.x; m < a.P; m += blockDim.x) tw[m] = twiddle<FF>(m, a.P, a.sign);
  for (int m = threadIdx.x; m < a.P1; m += blockDim.x) t1[m] = twiddle<FF>(m * a.P2, a.P, a.sign);
  for (int m = threadIdx.x; m < a.P2; m += blockDim.x) t2[m] = twiddle<FF>(m * a.P1, a.P, a.sign);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const V zero = dzero<FF>();
  const S* in = reinterpret_cast<const S*>(a.in);

  // copies of tile t's inputs into stage buf (one commit group per tile)
  auto issue = [&](int64_t t, int buf) {
    const int64_t it = t % a.tiles_i, og = t / a.tiles_i;
    const int o2 = (int)(og % a.O2), o1 = (int)(og / a.O2);
    const int64_t i0 = it * TI;
    const int64_t bin = o1 * a.a1 + o2 * a.a2 + i0;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage + buf * per_stage);
    for (int64_t e = threadIdx.x; e < per_stage; e += blockDim.x) {
      const int64_t j = e / TI, ii = e - j * TI;
      const bool ok = i0 + ii < a.I;
      cp_async_val<sizeof(S)>(sbase + (uint32_t)(e * sizeof(S)), ok ? in + bin + j * a.aj + ii : in,
                              ok ? (int)sizeof(S) : 0);
    }
  };

  int buf = 0;
  if ((int64_t)blockIdx.x < a.tiles) issue(blockIdx.x, 0);
  cp_async_commit_group();
  for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < a.tiles) issue(tn, buf ^ 1);
    cp_async_commit_group();
    cp_async_wait_group<1>();   // this tile's copies have landed
    __syncthreads();
    const int64_t it = t % a.tiles_i, og = t / a.tiles_i;
    const int o2 = (int)(og % a.O2), o1 = (int)(og / a.O2);
    const int64_t i0 = it * TI;
    const int64_t bout = o1 * a.b1 + o2 * a.b2;
    const S* st = stage + buf * per_stage;
    // stage A: items (sub, n2)
    for (int item = warp; item < a.nsub * a.P2; item += nw) {
      const int sub = item / a.P2, n2 = item - sub * a.P2;
      const int64_t ii = (int64_t)sub * 32 + lane;
      const int64_t i = i0 + ii;
      const bool ok = i < a.I;
      const int nin = min(a.P1, (a.Pin - n2 + a.P2 - 1) / a.P2);   // n1 with P2 n1 + n2 < Pin
      V x[DFT_R];
#pragma unroll
      for (int n1 = 0; n1 < DFT_R; ++n1) {
        x[n1] = zero;
        if (n1 < nin) x[n1] = from_stored<IN, FF>(st[(int64_t)(a.P2 * n1 + n2) * TI + ii]);
      }
      if (a.P2 == 1) {
        // direct sum: the outputs go straight to global memory
#pragma unroll 1
        for (int k1 = 0; k1 < a.Pout; ++k1) {
          const V v = short_dft<FF>(x, t1, nin, k1, a.P1);
          if (ok) dstore<FF, OUT>(a.out, bout + (int64_t)k1 * a.bf + i, v, a.scale, a.accumulate);
        }
      } else {
        V* Ys = Y + (int64_t)sub * a.P * 32 + lane;
#pragma unroll 1
        for (int k1 = 0; k1 < a.P1; ++k1) {
          const V v = short_dft<FF>(x, t1, nin, k1, a.P1);
          Ys[(n2 * a.P1 + k1) * 32] = n2 * k1 == 0 ? v : dmul<FF>(v, tw[n2 * k1]);   // n2 k1 < P
        }
      }
    }
    if (a.P2 > 1) {
      __syncthreads();
      // stage B: items (sub, k1)
      for (int item = warp; item < a.nsub * a.P1; item += nw) {
        const int sub = item / a.P1, k1 = item - sub * a.P1;
        if (k1 >= a.Pout) continue;
        const int64_t i = i0 + sub * 32 + lane;
        const bool ok = i < a.I;
        const V* Ys = Y + (int64_t)sub * a.P * 32 + lane;
        V y[DFT_R];
#pragma unroll
        for (int n2 = 0; n2 < DFT_R; ++n2) y[n2] = n2 < a.P2 ? Ys[(n2 * a.P1 + k1) * 32] : zero;
#pragma unroll 1
        for (int k2 = 0; k2 < a.P2; ++k2) {
          const int f = k1 + a.P1 * k2;
          if (f >= a.Pout) break;
          const V v = short_dft<FF>(y, t2, a.P2, k2, a.P2);
          if (ok) dstore<FF, OUT>(a.out, bout + (int64_t)f * a.bf + i, v, a.scale, a.accumulate);
        }
      }
    }
    __syncthreads();   // Y and this stage are free for the next tiles
    buf ^= 1;
  }
  cp_async_wait_group<0>();
}

// Direct form for short input lines: one thread per (line, inner index)
// loads its Pin inputs into registers (all loads in flight at once, 32
// consecutive inner indices per warp) and forms every kept output as a
// direct sum, with no shared-memory exchange and no barrier.  Pin * Pout
// multiply-adds per line: the choice for FP32 arithmetic (cheap next to the
// bytes it moves) and for float-float lines of a prime length.
template <bool FF, int IN, int OUT, int MAXIN>
__global__ void __launch_bounds__(256) k_dft_direct(const DftArgs a) {
  using V = DVal<FF>;
  using S = typename DIn<IN>::T;
  extern __shared__ __align__(16) unsigned char dsm[];
  V* tw = reinterpret_cast<V*>(dsm);   // w^m, m < P
  V* tf = tw + a.P;                    // w^{(f j) mod P} at f Pin + j: no index arithmetic in the sums
  for (int m = threadIdx.x; m < a.P; m += blockDim.x) tw[m] = twiddle<FF>(m, a.P, a.sign);
  __syncthreads();
  for (int e = threadIdx.x; e < a.Pout * a.Pin; e += blockDim.x) {
    const int f = e / a.Pin, j = e - f * a.Pin;
    tf[e] = tw[(f * j) % a.P];
  }
  __syncthreads();
  const S* in = reinterpret_cast<const S*>(a.in);
  const V zero = dzero<FF>();
  const int64_t items = (int64_t)a.O1 * a.O2 * a.I;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g % a.I, og = g / a.I;
    const int o2 = (int)(og % a.O2), o1 = (int)(og / a.O2);
    const S* src = in + o1 * a.a1 + o2 * a.a2 + i;
    V x[MAXIN];
#pragma unroll
    for (int j = 0; j < MAXIN; ++j) x[j] = j < a.Pin ? from_stored<IN, FF>(src[(int64_t)j * a.aj]) : zero;
    const int64_t dst = o1 * a.b1 + o2 * a.b2 + i;
    int64_t rowbase = 0, col = 0;
    if constexpr (OUT == DFT_BF16R) {
      const int64_t ib = i / a.row_b;
      rowbase = o1 * a.b1r + o2 * a.b2r + ib;
      col = i - ib * a.row_b;
    }
#pragma unroll 1
    for (int f = 0; f < a.Pout; ++f) {
      const V* tr = tf + f * a.Pin;
      V v;
      if constexpr (FF) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll
        for (int j = 0; j < MAXIN; ++j)
          if (j < a.Pin) ff_cmac(tr[j], x[j], rh, rl, ih, il);
        v = ff_norm(rh, rl, ih, il);
      } else {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < MAXIN; ++j)
          if (j < a.Pin) {
            const float2 t = tr[j];
            re = fmaf(t.x, x[j].x, fmaf(-t.y, x[j].y, re));
            im = fmaf(t.x, x[j].y, fmaf(t.y, x[j].x, im));
          }
        v = make_float2(re, im);
      }
      if constexpr (OUT == DFT_BF16R)
        store_bf16r(a, rowbase, col, f, v);
      else
        dstore<FF, OUT>(a.out, dst + (int64_t)f * a.bf, v, a.scale, a.accumulate);
    }
  }
}

// FP32 passes of a power-of-two length P <= 32: the whole line in
// registers (zeros past Pin) and log2 P radix-2 decimation-in-frequency
// stages, which leave X_f in bit-reversed order: register k holds X_f with
// f the LG-bit reversal of k, and the first Pout are stored.  P/2 log2 P
// butterflies per line against Pin Pout complex multiply-adds of the direct
// form (80 against 512 for the 16 -> 32 forward pass).  Twiddles w^m from
// shared memory (broadcast reads); every register index is a compile-time
// constant.
__host__ __device__ constexpr int ilog2(int p) { return p <= 1 ? 0 : 1 + ilog2(p / 2); }

template <int IN, int OUT, int P>
__global__ void __launch_bounds__(256) k_dft_fft2(const DftArgs a) {
  static_assert(P >= 2 && P <= 32 && (P & (P - 1)) == 0, "radix-2 lengths 2..32");
  constexpr int LG = ilog2(P);
  using S = typename DIn<IN>::T;
  __shared__ float2 tw[P];   // w^m, m < P
  for (int m = threadIdx.x; m < P; m += blockDim.x) tw[m] = twiddle<false>(m, P, a.sign);
  __syncthreads();
  const S* in = reinterpret_cast<const S*>(a.in);
  const int64_t items = (int64_t)a.O1 * a.O2 * a.I;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g % a.I, og = g / a.I;
    const int o2 = (int)(og % a.O2), o1 = (int)(og / a.O2);
    const S* src = in + o1 * a.a1 + o2 * a.a2 + i;
    float2 v[P];
#pragma unroll
    for (int j = 0; j < P; ++j)
      v[j] = j < a.Pin ? from_stored<IN, false>(src[(int64_t)j * a.aj]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int sg = 0; sg < LG; ++sg) {
      const int h = P >> (sg + 1), m = 2 * h, step = 1 << sg;   // span m, twiddle w^(t step)
#pragma unroll
      for (int k = 0; k < P; k += m)
#pragma unroll
        for (int t = 0; t < h; ++t) {
          const float2 u = v[k + t], x = v[k + t + h];
          v[k + t] = make_float2(u.x + x.x, u.y + x.y);
          float2 d = make_float2(u.x - x.x, u.y - x.y);
          if (t != 0) {
            const float2 w = tw[t * step];
            d = make_float2(fmaf(w.x, d.x, -w.y * d.y), fmaf(w.x, d.y, w.y * d.x));
          }
          v[k + t + h] = d;
        }
    }
    const int64_t dst = o1 * a.b1 + o2 * a.b2 + i;
    int64_t rowbase = 0, col = 0;
    if constexpr (OUT == DFT_BF16R) {
      const int64_t ib = i / a.row_b;
      rowbase = o1 * a.b1r + o2 * a.b2r + ib;
      col = i - ib * a.row_b;
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int f = (int)(__brev((unsigned)k) >> (32 - LG));
      if (f < a.Pout) {
        if constexpr (OUT == DFT_BF16R)
          store_bf16r(a, rowbase, col, f, v[k]);
        else
          dstore<false, OUT>(a.out, dst + (int64_t)f * a.bf, v[k], a.scale, a.accumulate);
      }
    }
  }
}

template <int IN, int OUT>
fmpb_status launch_fft2(const char* name, const DftArgs& a, cudaStream_t st) {
  const int64_t items = (int64_t)a.O1 * a.O2 * a.I;
  int sms = 0, dev = 0;
  FMPB_CUDA(cudaGetDevice(&dev));
  FMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  auto go = [&](auto kern) -> fmpb_status {
    int per_sm = 0;
    FMPB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
    const int64_t grid = std::min<int64_t>((items + 255) / 256, (int64_t)std::max(1, per_sm) * sms * DFT_WAVES);
    FMPB_LAUNCH(name, st, kern<<<(unsigned)grid, 256, 0, st>>>(a));
    FMPB_CUDA(cudaGetLastError());
    return FMPB_OK;
  };
  switch (a.P) {
    case 8: return go(k_dft_fft2<IN, OUT, 8>);
    case 16: return go(k_dft_fft2<IN, OUT, 16>);
    case 32: return go(k_dft_fft2<IN, OUT, 32>);
    default: break;
  }
  set_error("dft_pass: no radix-2 pass of length %d", a.P);
  return FMPB_EINVAL;
}

// complex multiply-adds of a plan (stage A + twiddles + stage B)
int64_t plan_cost(int P, int Pin, int Pout, int P1) {
  const int P2 = P / P1;
  if (P2 == 1) return (int64_t)Pin * Pout;
  return (int64_t)Pin * P1 + P + (int64_t)Pout * P2;
}

// Largest dynamic shared memory a two-factor pass may ask for.
constexpr int DFT_MAX_SMEM = 200 * 1024;
template <bool FF, int IN, int OUT>
fmpb_status launch_dft(const char* name, const DftArgs& a, size_t smem, int threads, cudaStream_t st) {
  FMPB_CUDA((smem_limit_once<k_dft<FF, IN, OUT>>(DFT_MAX_SMEM)));
  // CTAs walking their share of the tiles, DFT_WAVES times as many as can be
  // resident: few enough to amortise the twiddle set-up, short-lived enough
  // that a pass run beside another stream's kernels frees SM slots often
  int per_sm = 0, sms = 0, dev = 0;
  FMPB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dft<FF, IN, OUT>, threads, smem));
  FMPB_CUDA(cudaGetDevice(&dev));
  FMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = std::min<int64_t>(a.tiles, (int64_t)std::max(1, per_sm) * sms * DFT_WAVES);
  FMPB_LAUNCH(name, st, k_dft<FF, IN, OUT><<<(unsigned)grid, threads, smem, st>>>(a));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

template <bool FF, int IN, int OUT>
fmpb_status launch_direct(const char* name, const DftArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.P + a.Pout * a.Pin) * (FF ? sizeof(float4) : sizeof(float2));
  const int64_t items = (int64_t)a.O1 * a.O2 * a.I;
  int sms = 0, dev = 0;
  FMPB_CUDA(cudaGetDevice(&dev));
  FMPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  auto go = [&](auto kern) -> fmpb_status {
    int per_sm = 0;
    FMPB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
    const int64_t grid = std::min<int64_t>((items + 255) / 256, (int64_t)std::max(1, per_sm) * sms * DFT_WAVES);
    FMPB_LAUNCH(name, st, kern<<<(unsigned)grid, 256, smem, st>>>(a));
    FMPB_CUDA(cudaGetLastError());
    return FMPB_OK;
  };
  if (a.Pin <= 8) return go(k_dft_direct<FF, IN, OUT, 8>);
  if (a.Pin <= 16) return go(k_dft_direct<FF, IN, OUT, 16>);
  return go(k_dft_direct<FF, IN, OUT, 32>);
}

}  // namespace

bool dft_plan(int P, int Pin, int Pout, int* P1out) {
  int best = 0;
  int64_t cost = 0;
  for (int p1 = 1; p1 <= DFT_R && p1 <= P; ++p1) {
    if (P % p1 || P / p1 > DFT_R) continue;
    const int64_t c = plan_cost(P, Pin, Pout, p1);
    if (!best || c < cost) {
      best = p1;
      cost = c;
    }
  }
  if (!best) return false;
  *P1out = best;
  return true;
}

bool dft_supported(int P) {
  int p1;
  return P <= 1 || dft_plan(P, P, P, &p1);
}

// One plan of a pass: kind 0 = the direct form, kind 1 = the two-factor
// form with the split P1, kind 2 = the radix-2 form (FP32, P a power of two
// up to 32).
struct DftPlan {
  int kind, P1;
};
bool fft2_ok(bool ff_arith, int P) { return !ff_arith && (P == 8 || P == 16 || P == 32); }
const char* plan_name(int kind) { return kind == 0 ? "direct" : (kind == 1 ? "split" : "fft2_"); }

static fmpb_status run_plan(const char* name, const DftPlan& plan, bool ff_arith, int in_fmt, int out_fmt,
                            DftArgs a, cudaStream_t st) {
  const int P = a.P, Pin = a.Pin;
  const int64_t I = a.I;
  const int O1 = a.O1, O2 = a.O2;
  a.P1 = plan.kind == 1 ? plan.P1 : P;
  a.P2 = P / a.P1;
  if (plan.kind == 2) {
    if (in_fmt == DFT_F32 && out_fmt == DFT_BF16R) return launch_fft2<DFT_F32, DFT_BF16R>(name, a, st);
    if (in_fmt == DFT_CD && out_fmt == DFT_BF16R) return launch_fft2<DFT_CD, DFT_BF16R>(name, a, st);
    if (in_fmt == DFT_CD && out_fmt == DFT_F32) return launch_fft2<DFT_CD, DFT_F32>(name, a, st);
    if (in_fmt == DFT_F32 && out_fmt == DFT_F32) return launch_fft2<DFT_F32, DFT_F32>(name, a, st);
    if (in_fmt == DFT_F32 && out_fmt == DFT_CD) return launch_fft2<DFT_F32, DFT_CD>(name, a, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_F32) return launch_fft2<DFT_FF, DFT_F32>(name, a, st);
    set_error("dft_pass: unsupported storage formats %d -> %d", in_fmt, out_fmt);
    return FMPB_EINVAL;
  }
  if (plan.kind == 0) {
    if (ff_arith) {
      if (in_fmt == DFT_CD && out_fmt == DFT_FF) return launch_direct<true, DFT_CD, DFT_FF>(name, a, st);
      if (in_fmt == DFT_FF && out_fmt == DFT_FF) return launch_direct<true, DFT_FF, DFT_FF>(name, a, st);
      if (in_fmt == DFT_FF && out_fmt == DFT_CD) return launch_direct<true, DFT_FF, DFT_CD>(name, a, st);
      if (in_fmt == DFT_CD && out_fmt == DFT_CD) return launch_direct<true, DFT_CD, DFT_CD>(name, a, st);
    } else {
      if (in_fmt == DFT_F32 && out_fmt == DFT_BF16R) return launch_direct<false, DFT_F32, DFT_BF16R>(name, a, st);
      if (in_fmt == DFT_CD && out_fmt == DFT_BF16R) return launch_direct<false, DFT_CD, DFT_BF16R>(name, a, st);
      if (in_fmt == DFT_CD && out_fmt == DFT_F32) return launch_direct<false, DFT_CD, DFT_F32>(name, a, st);
      if (in_fmt == DFT_F32 && out_fmt == DFT_F32) return launch_direct<false, DFT_F32, DFT_F32>(name, a, st);
      if (in_fmt == DFT_F32 && out_fmt == DFT_CD) return launch_direct<false, DFT_F32, DFT_CD>(name, a, st);
      if (in_fmt == DFT_FF && out_fmt == DFT_F32) return launch_direct<false, DFT_FF, DFT_F32>(name, a, st);
    }
    set_error("dft_pass: unsupported storage formats %d -> %d", in_fmt, out_fmt);
    return FMPB_EINVAL;
  }
  const size_t vb = ff_arith ? sizeof(float4) : sizeof(float2);
  const size_t sb = in_fmt == DFT_F32 ? sizeof(float2) : sizeof(float4);
  // inner sub-tiles of 32 per CTA: enough items for up to 8 warps in both
  // stages, within the inner extent and the shared-memory budget, then fewer
  // while the grid would leave SMs idle (small passes are latency-bound)
  const int mn = std::min(a.P1, a.P2);
  int nsub = std::max(1, std::min(8, (8 + mn - 1) / mn));
  nsub = (int)std::min<int64_t>(nsub, (I + 31) / 32);
  auto smem_for = [&](int ns) {
    const size_t head = (size_t)(P + a.P1 + a.P2 + (a.P2 > 1 ? (size_t)ns * P * 32 : 0)) * vb;
    return (head + 15) / 16 * 16 + 2 * (size_t)Pin * 32 * ns * sb;
  };
  while (nsub > 1 && smem_for(nsub) > 72 * 1024) --nsub;
  auto tiles_for = [&](int ns) { return (I + 32 * ns - 1) / (32 * ns) * O1 * O2; };
  while (nsub > 1 && tiles_for(nsub) < 4 * 152) --nsub;
  a.nsub = nsub;
  a.tiles_i = (I + 32 * nsub - 1) / (32 * nsub);
  a.tiles = a.tiles_i * O1 * O2;
  const size_t smem = smem_for(nsub);
  if (smem > (size_t)DFT_MAX_SMEM) {
    set_error("dft_pass: axis length %d too large", P);
    return FMPB_EINVAL;
  }
  const int warps = std::max(1, std::min(DFT_THREADS / 32, std::max(nsub * a.P2, a.P2 > 1 ? nsub * a.P1 : 0)));
  const int threads = 32 * warps;
  if (ff_arith) {
    if (in_fmt == DFT_CD && out_fmt == DFT_FF) return launch_dft<true, DFT_CD, DFT_FF>(name, a, smem, threads, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_FF) return launch_dft<true, DFT_FF, DFT_FF>(name, a, smem, threads, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_CD) return launch_dft<true, DFT_FF, DFT_CD>(name, a, smem, threads, st);
    if (in_fmt == DFT_CD && out_fmt == DFT_CD) return launch_dft<true, DFT_CD, DFT_CD>(name, a, smem, threads, st);
  } else {
    if (in_fmt == DFT_CD && out_fmt == DFT_F32) return launch_dft<false, DFT_CD, DFT_F32>(name, a, smem, threads, st);
    if (in_fmt == DFT_F32 && out_fmt == DFT_F32) return launch_dft<false, DFT_F32, DFT_F32>(name, a, smem, threads, st);
    if (in_fmt == DFT_F32 && out_fmt == DFT_CD) return launch_dft<false, DFT_F32, DFT_CD>(name, a, smem, threads, st);
    if (in_fmt == DFT_FF && out_fmt == DFT_F32) return launch_dft<false, DFT_FF, DFT_F32>(name, a, smem, threads, st);
  }
  set_error("dft_pass: unsupported storage formats %d -> %d", in_fmt, out_fmt);
  return FMPB_EINVAL;
}

// DFT-pass autotuner: the first out-of-place, non-accumulating call of a
// pass shape times every candidate plan (the direct form where the inputs
// fit the registers, the two-factor form for every split into factors of at
// most 16) with CUDA events on the caller's stream, after one untimed launch
// each, keeps the fastest and runs it once more, so that the output carries
// the chosen plan's rounding on the first call as on every later one.  In-place and accumulating passes, passes inside
// a stream capture and shapes with one candidate take the model's plan
// (fewest multiply-adds; the direct form for FP32 lines of at most 32
// inputs).
// The key is the line shape and arithmetic only: every later pass of that
// shape, whatever its inner extent and line count, takes the plan its first
// timed pass chose, so that operators batched together round exactly as
// they do alone (the inner extent and line count of that first pass are
// kept for the summary).
struct DftKey {
  int dev, ff, in, out, P, Pin, Pout;
  int64_t I, lines;
  bool operator<(const DftKey& o) const {
    return std::tie(dev, ff, in, out, P, Pin, Pout) < std::tie(o.dev, o.ff, o.in, o.out, o.P, o.Pin, o.Pout);
  }
};
struct DftTuned {
  DftPlan plan;
  int n;
  DftPlan cand[DFT_R + 2];
  float ms[DFT_R + 2];
};
std::mutex g_dft_mu;
std::map<DftKey, DftTuned> g_dft_tune;
int g_dft_forced = -1;   // >= 0: fmpb_set_dft_plan override (plan kind)

bool dft_rows_ok(int P, int Pin) { return Pin <= 32 || fft2_ok(false, P); }

fmpb_status dft_pass(const char* name, bool ff_arith, int in_fmt, int out_fmt, const void* in, void* out, int O1,
                     int O2, int64_t I, int64_t a1, int64_t a2, int64_t aj, int64_t b1, int64_t b2, int64_t bf,
                     int Pin, int Pout, int P, int sign, double scale, bool accumulate, cudaStream_t st,
                     int64_t row_b, int row_kh) {
  const bool rows = out_fmt == DFT_BF16R;
  if (rows && (ff_arith || accumulate || row_b < 1 || row_kh < row_b || b1 % row_b || b2 % row_b || bf % row_b ||
               !dft_rows_ok(P, Pin))) {
    set_error("dft_pass: BF16 rows take an FP32 direct or radix-2 pass whose output strides are whole rows");
    return FMPB_EINVAL;
  }
  int P1 = 0;
  if (!dft_plan(P, Pin, Pout, &P1)) {
    set_error("dft_pass: axis length %d has no split into two factors of at most %d", P, DFT_R);
    return FMPB_EINVAL;
  }
  if (Pin < 1 || Pin > P || Pout < 1 || Pout > P || O1 < 1 || O2 < 1 || I < 1) {
    set_error("dft_pass: bad line geometry (Pin %d, Pout %d, P %d)", Pin, Pout, P);
    return FMPB_EINVAL;
  }
  if (accumulate && out_fmt != DFT_CD) {
    set_error("dft_pass: accumulation needs complex-double output");
    return FMPB_EINVAL;
  }
  DftArgs a{};
  a.in = in;
  a.out = out;
  a.I = I;
  a.a1 = a1;
  a.a2 = a2;
  a.aj = aj;
  a.b1 = b1;
  a.b2 = b2;
  a.bf = bf;
  a.O1 = O1;
  a.O2 = O2;
  a.Pin = Pin;
  a.Pout = Pout;
  a.P = P;
  a.sign = sign;
  a.accumulate = accumulate ? 1 : 0;
  a.scale = scale;
  if (rows) {
    a.row_b = row_b;
    a.row_kh = row_kh;
    a.b1r = b1 / row_b;
    a.b2r = b2 / row_b;
    a.bfr = bf / row_b;
  }
  // the model's plan
  const bool direct_ok = ff_arith ? Pin <= 16 : Pin <= 32;
  DftPlan model{1, P1};
  if (ff_arith ? (P / P1 == 1 && direct_ok) : direct_ok) model = DftPlan{0, P};
  if (P / P1 == 1 && !direct_ok) model = DftPlan{1, P1};
  // candidates
  DftPlan cand[DFT_R + 2];
  int nc = 0;
  if (direct_ok) cand[nc++] = DftPlan{0, P};
  if (fft2_ok(ff_arith, P)) cand[nc++] = DftPlan{2, P};
  for (int p1 = 2; p1 <= DFT_R && p1 < P && !rows; ++p1)
    if (P % p1 == 0 && P / p1 <= DFT_R && nc <= DFT_R) cand[nc++] = DftPlan{1, p1};
  if (rows) model = direct_ok ? DftPlan{0, P} : DftPlan{2, P};
  int forced = -1;
  {
    std::lock_guard<std::mutex> lk(g_dft_mu);
    forced = g_dft_forced;
  }
  if (forced >= 0) {
    // the requested kind where the pass has it, else the model's plan
    DftPlan f = model;
    if (forced == 0 && direct_ok) f = DftPlan{0, P};
    if (forced == 1 && P / P1 > 1 && !rows) f = DftPlan{1, P1};
    if (forced == 2 && fft2_ok(ff_arith, P)) f = DftPlan{2, P};
    return run_plan(name, f, ff_arith, in_fmt, out_fmt, a, st);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FMPB_CUDA(cudaStreamIsCapturing(st, &cap));
  if (in == out || accumulate || cap != cudaStreamCaptureStatusNone || nc < 2)
    return run_plan(name, model, ff_arith, in_fmt, out_fmt, a, st);
  int dev = 0;
  FMPB_CUDA(cudaGetDevice(&dev));
  const DftKey key{dev, ff_arith ? 1 : 0, in_fmt, out_fmt, P, Pin, Pout, I, (int64_t)O1 * O2};
  {
    std::lock_guard<std::mutex> lk(g_dft_mu);
    auto it = g_dft_tune.find(key);
    if (it != g_dft_tune.end()) {
      const DftPlan chosen = it->second.plan;
      return run_plan(name, chosen, ff_arith, in_fmt, out_fmt, a, st);
    }
  }
  DftTuned tuned{};
  tuned.n = nc;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  fmpb_status s = FMPB_OK;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "dft tuning events");
  float best = 1e30f;
  DftPlan chosen = model;
  for (int c = 0; c < nc && s == FMPB_OK; ++c) {
    tuned.cand[c] = cand[c];
    s = run_plan(name, cand[c], ff_arith, in_fmt, out_fmt, a, st);
    if (s == FMPB_OK && cudaEventRecord(t0, st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "dft tuning");
    if (s == FMPB_OK) s = run_plan(name, cand[c], ff_arith, in_fmt, out_fmt, a, st);
    if (s == FMPB_OK && (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess))
      s = cuda_status(cudaGetLastError(), "dft tuning");
    float ms = 0.f;
    if (s == FMPB_OK && cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) s = cuda_status(cudaGetLastError(), "dft tuning");
    tuned.ms[c] = ms;
    if (s == FMPB_OK && ms < best) {
      best = ms;
      chosen = cand[c];
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (s != FMPB_OK) return s;
  tuned.plan = chosen;
  {
    std::lock_guard<std::mutex> lk(g_dft_mu);
    g_dft_tune[key] = tuned;
  }
  // the chosen plan writes the output last, so that the first call of a
  // shape gives the same rounding as every later one
  return run_plan(name, chosen, ff_arith, in_fmt, out_fmt, a, st);
}

fmpb_status dft_force_plan(int kind) {
  if (kind < -1 || kind > 2) {
    set_error("set_dft_plan: plan kind %d outside -1..2", kind);
    return FMPB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_dft_mu);
  g_dft_forced = kind;
  return FMPB_OK;
}

void dft_tuning_summary(std::string& out) {
  std::lock_guard<std::mutex> lk(g_dft_mu);
  char buf[256];
  for (const auto& kv : g_dft_tune) {
    const DftKey& k = kv.first;
    const DftTuned& t = kv.second;
    int n = snprintf(buf, sizeof(buf),
                     "%s{\"kernel\": \"dft\", \"device\": %d, \"arith\": \"%s\", \"P\": %d, \"Pin\": %d, "
                     "\"Pout\": %d, \"inner\": %lld, \"lines\": %lld, \"chosen\": \"%s%d\", \"ms\": {",
                     out.size() > 1 ? ", " : "", k.dev, k.ff ? "ff" : "f32", k.P, k.Pin, k.Pout, (long long)k.I,
                     (long long)k.lines, plan_name(t.plan.kind), t.plan.kind == 1 ? t.plan.P1 : k.P);
    out.append(buf, n);
    for (int c = 0; c < t.n; ++c) {
      n = snprintf(buf, sizeof(buf), "%s\"%s%d\": %.4f", c ? ", " : "", plan_name(t.cand[c].kind),
                   t.cand[c].kind == 1 ? t.cand[c].P1 : k.P, t.ms[c]);
      out.append(buf, n);
    }
    out += "}}";
  }
}

}  // namespace fmpb

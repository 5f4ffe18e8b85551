// Restarted GMRES for R independent right-hand sides sharing each product
// (Sec. 4: the systems of Eqs. (toeplitzBEM) and (FMPBEMsystem) are solved by
// GMRES with a relative residual tolerance).  Everything lives on the device:
// the Krylov basis as float-float pairs (48-bit significand; FP32 values for
// the BF16 inner solves), the product vectors, Hessenberg columns, rotations
// and least-squares update in FP64 (the stored rotations applied to a new
// column in float-float, as a scan).  The Arnoldi step is DCGS2, classical
// Gram-Schmidt whose reorthogonalising second pass is folded into the next
// step's projections (one dots and one update pass over the basis per step),
// where the operator multiplies basis vectors directly (float-float or FP32)
// and the raw Hessenberg copy fits; otherwise classical Gram-Schmidt
// with a second pass whenever the first one removed more than half of
// ||w||^2 (Kahan-Parlett "twice is enough").  The host sequences launches,
// reads the convergence flags and residual estimates every few iterations
// (the only device to host traffic; next_block sets the cadence) and enforces
// the wall-clock limit between launches: no kernel waits on anything.
#include <chrono>
#include <functional>

#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "gmres.cuh"
#include "ff.cuh"

namespace fmpb {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 64;   // upper bound on partial sums per (vector, rhs)
constexpr int MAX_RESTART = 1000;

// partial[(v*R + r)*gridDim.x + blk] = sum over the block's rows of
// conj(V_v[r]) w[r]; four independent accumulators per thread keep several
// loads in flight.
__global__ void k_dots(const cd* __restrict__ V, int64_t vstride, int nvec, const cd* __restrict__ w, int R,
                       int64_t N, cd* __restrict__ partial, const int* __restrict__ active) {
  const int blk = blockIdx.x, v = blockIdx.y, r = blockIdx.z;
  __shared__ double sre[RED_THREADS], sim[RED_THREADS];
  double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
  if (active[r]) {
    const cd* a = V + (int64_t)v * vstride + (int64_t)r * N;
    const cd* b = w + (int64_t)r * N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < N; i += 4 * stride) {
      cd x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = a[i + u * stride];
        y[u] = b[i + u * stride];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        re[u] = fma(x[u].x, y[u].x, fma(x[u].y, y[u].y, re[u]));
        im[u] = fma(x[u].x, y[u].y, fma(-x[u].y, y[u].x, im[u]));
      }
    }
    for (; i < N; i += stride) {
      cd x = a[i], y = b[i];
      re[0] = fma(x.x, y.x, fma(x.y, y.y, re[0]));
      im[0] = fma(x.x, y.y, fma(-x.y, y.x, im[0]));
    }
  }
  sre[threadIdx.x] = (re[0] + re[1]) + (re[2] + re[3]);
  sim[threadIdx.x] = (im[0] + im[1]) + (im[2] + im[3]);
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sre[threadIdx.x] += sre[threadIdx.x + s];
      sim[threadIdx.x] += sim[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[((int64_t)v * R + r) * gridDim.x + blk] = mkc(sre[0], sim[0]);
}

// out[v*R + r] (+)= sum_blk partial  (fixed order: deterministic)
__global__ void k_reduce_partials(const cd* __restrict__ partial, int nblk, int count, cd* __restrict__ out,
                                  int accumulate) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  cd s = mkc(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = cadd(s, partial[(int64_t)t * nblk + b]);
  out[t] = accumulate ? cadd(out[t], s) : s;
}

// y = b - y  (residual from a product)
__global__ void k_residual(const cd* __restrict__ b, cd* __restrict__ y, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = csub(b[i], y[i]);
}

// Per-RHS control state of one restart cycle.
struct GmresState {
  cd* H;           // R x (m+1) x m, column-major per rhs: H[r][j][i] at (r*m + j)*(m+1) + i
  double* cs;      // R x m
  cd* sn;          // R x m
  cd* g;           // R x (m+1)
  double* beta;    // R: ||r0||
  double* inv;     // R: 1 / norm (scratch for k_scale)
  double* bnorm;   // R
  double* resid;   // R: current residual estimate / ||b||
  int* active;     // R
  int* jcount;     // R: Arnoldi columns completed this cycle
  int* iters;      // R: Arnoldi steps taken while active (whole solve)
};

// Norms: sqrt(real(dot)) from the reduced dots.
__global__ void k_sqrt_real(const cd* __restrict__ d, double* __restrict__ out, double* __restrict__ inv, int R) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double v = sqrt(fmax(d[r].x, 0.0));
  out[r] = v;
  if (inv) inv[r] = v > 0.0 ? 1.0 / v : 0.0;
}

// Start of a cycle: g = (beta, 0...), resid = beta / bnorm, active = resid > tol.
__global__ void k_cycle_start(GmresState s, int R, int m, double tol) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  for (int i = 0; i <= m; ++i) s.g[r * (m + 1) + i] = mkc(0.0, 0.0);
  s.g[r * (m + 1)] = mkc(s.beta[r], 0.0);
  double rel = s.bnorm[r] > 0.0 ? s.beta[r] / s.bnorm[r] : 0.0;
  s.resid[r] = rel;
  s.active[r] = (rel > tol && s.beta[r] > 0.0) ? 1 : 0;
  s.jcount[r] = 0;
}

// Column j of H from the projections h (nvec = j+1) and the norm of w;
// applies the previous rotations, forms the new one, updates g and the
// residual estimate.  One warp per rhs: the lanes stage the column and the
// rotations in shared memory as float-float values, lane 0 runs the
// sequential recurrence in float-float arithmetic on the FP32 pipe (GB300's
// FP64 latency would make this chain of up to 1,000 dependent rotations the
// slowest step of an iteration), and the new rotation, g and the residual
// estimate are formed in FP64.
__device__ __forceinline__ ffc ffc_from_cd(cd v) { return {ff_from_d(v.x), ff_from_d(v.y)}; }
__device__ __forceinline__ cd ffc_to_cd(ffc v) { return mkc(ff_to_d(v.re), ff_to_d(v.im)); }
__device__ __forceinline__ ffc ffc_add(ffc a, ffc b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ ffc ffc_sub(ffc a, ffc b) { return {ff_sub(a.re, b.re), ff_sub(a.im, b.im)}; }
__device__ __forceinline__ ffc ffc_scale(ffc a, ff c) { return {ff_mul(a.re, c), ff_mul(a.im, c)}; }
__device__ __forceinline__ ffc ffc_conj(ffc a) { return {a.re, ff_neg(a.im)}; }
__device__ __forceinline__ ffc ffc_neg(ffc a) { return {ff_neg(a.re), ff_neg(a.im)}; }
__device__ __forceinline__ ffc ffc_shfl_up(ffc a, int off) {
  return {{__shfl_up_sync(0xffffffffu, a.re.h, off), __shfl_up_sync(0xffffffffu, a.re.l, off)},
          {__shfl_up_sync(0xffffffffu, a.im.h, off), __shfl_up_sync(0xffffffffu, a.im.l, off)}};
}

constexpr int GIV_WARPS = 4;   // warps of a k_givens CTA (one CTA per system)
__global__ void __launch_bounds__(32 * GIV_WARPS) k_givens(GmresState s, const cd* __restrict__ h,
                                                           const double* __restrict__ wnorm, int R, int m, int j,
                                                           double tol) {
  const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NT = 32 * GIV_WARPS;
  if (!s.active[r]) return;
  if (tid == 0) s.iters[r] += 1;
  __shared__ ffc col[MAX_RESTART + 1];
  __shared__ ff csv[MAX_RESTART];
  __shared__ ffc snv[MAX_RESTART];
  __shared__ ffc wal[GIV_WARPS], wbe[GIV_WARPS];   // each warp's composed map
  for (int i = tid; i <= j; i += NT) col[i] = ffc_from_cd(h[i * R + r]);
  for (int i = tid; i < j; i += NT) {
    csv[i] = ff_from_d(s.cs[r * m + i]);
    snv[i] = ffc_from_cd(s.sn[r * m + i]);
  }
  __syncthreads();
  // [c  s; -conj(s) c] applied to (a_i, h_{i+1}) for i < j, a_0 = h_0: the
  // rotated entry is c_i a_i + s_i h_{i+1} and the carried one
  // a_{i+1} = -conj(s_i) a_i + c_i h_{i+1}, an affine recurrence.  Each of
  // the 128 threads composes the maps of one chunk of ceil(j/128) rotations;
  // a shuffle scan within each warp and the composed warp maps give every
  // thread the value entering its chunk, and each thread then rotates its
  // chunk: sequential depth about 2 j / 128 + 9 instead of j.
  cd* Hcol = s.H + ((int64_t)r * m + j) * (m + 1);
  __shared__ ffc carry;
  {
    const int L = (j + NT - 1) / NT;
    const int i0 = min(j, tid * L), i1 = min(j, i0 + L);
    const ffc one = {ff_make(1.f), ff_make(0.f)}, zero = {ff_make(0.f), ff_make(0.f)};
    ffc al = one, be = zero;   // chunk map z -> al z + be
    for (int i = i0; i < i1; ++i) {
      const ffc ai = ffc_neg(ffc_conj(snv[i]));
      be = ffc_add(ffc_mul(ai, be), ffc_scale(col[i + 1], csv[i]));
      al = ffc_mul(ai, al);
    }
    for (int off = 1; off < 32; off <<= 1) {   // inclusive scan within the warp: later map after earlier
      const ffc pa = ffc_shfl_up(al, off), pb = ffc_shfl_up(be, off);
      if (lane >= off) {
        be = ffc_add(ffc_mul(al, pb), be);
        al = ffc_mul(al, pa);
      }
    }
    if (lane == 31) {
      wal[warp] = al;
      wbe[warp] = be;
    }
    __syncthreads();
    // the value entering this warp: the maps of the warps before it applied to a_0
    ffc aw = col[0];
    for (int u = 0; u < warp; ++u) aw = ffc_add(ffc_mul(wal[u], aw), wbe[u]);
    const ffc pa = ffc_shfl_up(al, 1), pb = ffc_shfl_up(be, 1);
    ffc a = lane == 0 ? aw : ffc_add(ffc_mul(pa, aw), pb);
    for (int i = i0; i < i1; ++i) {
      const ff c = csv[i];
      const ffc sn = snv[i];
      const ffc b = col[i + 1];
      Hcol[i] = ffc_to_cd(ffc_add(ffc_scale(a, c), ffc_mul(sn, b)));
      a = ffc_sub(ffc_scale(b, c), ffc_mul(ffc_conj(sn), a));
    }
    if ((i0 < i1 && i1 == j) || (j == 0 && tid == 0)) carry = a;
  }
  __syncthreads();
  if (warp != 0) return;
  __shared__ cd top;
  if (lane == 0) {
    cd ad = ffc_to_cd(carry);
    const cd b = mkc(wnorm[r], 0.0);
    const double na = hypot(ad.x, ad.y), nb = hypot(b.x, b.y);
    double c;
    cd sn;
    if (nb == 0.0) {
      c = 1.0;
      sn = mkc(0.0, 0.0);
    } else if (na == 0.0) {
      c = 0.0;
      sn = mkc(1.0, 0.0);
      ad = mkc(0.0, 0.0);
    } else {
      const double t = hypot(na, nb);
      c = na / t;
      // sn = (a/|a|) conj(b) / t
      const cd ua = mkc(ad.x / na, ad.y / na);
      sn = cmulr(cmul(ua, cconj(b)), 1.0 / t);
    }
    s.cs[r * m + j] = c;
    s.sn[r * m + j] = sn;
    top = cadd(cmulr(ad, c), cmul(sn, b));
    cd* g = s.g + r * (m + 1);
    const cd gj = g[j];
    g[j] = cmulr(gj, c);
    g[j + 1] = cmul(mkc(-sn.x, sn.y), gj);   // -conj(sn) g_j
    s.jcount[r] = j + 1;
    const double rel = hypot(g[j + 1].x, g[j + 1].y) / s.bnorm[r];
    s.resid[r] = rel;
    if (rel <= tol || wnorm[r] == 0.0) s.active[r] = 0;
  }
  __syncwarp();
  if (lane == 0) {
    Hcol[j] = top;
    Hcol[j + 1] = mkc(0.0, 0.0);
  }
}

// Back substitution H y = g for the jcount[r] completed columns; y into g.
// One warp per rhs: the inner sums are split over the lanes.
__global__ void k_backsolve(GmresState s, int R, int m) {
  const int r = blockIdx.x, lane = threadIdx.x;
  const int J = s.jcount[r];
  cd* g = s.g + r * (m + 1);
  __shared__ cd y[MAX_RESTART + 1];
  for (int i = lane; i <= m; i += 32) y[i] = i < J ? g[i] : mkc(0.0, 0.0);
  __syncwarp();
  for (int i = J - 1; i >= 0; --i) {
    double re = 0.0, im = 0.0;
    for (int k = i + 1 + lane; k < J; k += 32) {
      const cd hk = s.H[((int64_t)r * m + k) * (m + 1) + i];
      const cd yk = y[k];
      re += hk.x * yk.x - hk.y * yk.y;
      im += hk.x * yk.y + hk.y * yk.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      const cd acc = mkc(y[i].x - re, y[i].y - im);
      const cd d = s.H[((int64_t)r * m + i) * (m + 1) + i];
      const double den = d.x * d.x + d.y * d.y;
      y[i] = den > 0.0 ? mkc((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den) : mkc(0.0, 0.0);
    }
    __syncwarp();
  }
  for (int i = lane; i <= m; i += 32) g[i] = i < J ? y[i] : mkc(0.0, 0.0);
}

// ----------------------------------------------- float-float Krylov basis --
// The basis vectors are stored as float-float pairs (16 bytes per complex
// entry, as complex double) and every Gram-Schmidt dot product and update
// runs in float-float arithmetic on the FP32 pipe (48-bit significands): on
// GB300 the FP64 pipe would bound these passes at 1/58 of the FP32 rate.
// Reductions across threads, the Hessenberg matrix, the rotations, the
// solution update and the true residual stay in FP64.

__device__ __forceinline__ float4 ff_conj(float4 v) { return make_float4(v.x, v.y, -v.z, -v.w); }

// partial[(v*R + r)*gridDim.x + blk] = sum over the block's rows of conj(V_v[r]) w[r],
// for DOT_VB basis vectors per CTA (v = blockIdx.y *
// DOT_VB + q, q < DOT_VB, v < nvec): each row of w is loaded once for all of
// them.  Per-thread sums are reduced across the warp in float-float (FP32
// pipe; GB300's FP64 pipe would bound this step), then across the warps in
// FP64, in a fixed order (deterministic).
constexpr int DOT_VB = 4;
__global__ void __launch_bounds__(RED_THREADS) k_dots_ff4(const float4* __restrict__ V, int64_t vstride, int nvec,
                                                          const float4* __restrict__ w, int R, int64_t N,
                                                          cd* __restrict__ partial, const int* __restrict__ active) {
  const int blk = blockIdx.x, v0 = blockIdx.y * DOT_VB, r = blockIdx.z;
  const int nq = min(DOT_VB, nvec - v0);
  float rh[DOT_VB], rl[DOT_VB], ih[DOT_VB], il[DOT_VB];
#pragma unroll
  for (int q = 0; q < DOT_VB; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
  if (active[r]) {
    const float4* a = V + (int64_t)v0 * vstride + (int64_t)r * N;
    const float4* b = w + (int64_t)r * N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < N; i += stride) {
      const float4 y = b[i];
      float4 x[DOT_VB];
#pragma unroll
      for (int q = 0; q < DOT_VB; ++q) x[q] = q < nq ? a[(int64_t)q * vstride + i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < DOT_VB; ++q) ff_cmac(ff_conj(x[q]), y, rh[q], rl[q], ih[q], il[q]);
    }
  }
  __shared__ float4 sh[RED_THREADS / 32][DOT_VB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < DOT_VB; ++q) {
    ff_warp_sum(rh[q], rl[q]);
    ff_warp_sum(ih[q], il[q]);
    if (lane == 0) sh[warp][q] = make_float4(rh[q], rl[q], ih[q], il[q]);
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    const int q = threadIdx.x;
    double re = 0.0, im = 0.0;
    for (int u = 0; u < RED_THREADS / 32; ++u) {
      const float4 t = sh[u][q];
      re += (double)t.x + (double)t.y;
      im += (double)t.z + (double)t.w;
    }
    partial[((int64_t)(v0 + q) * R + r) * gridDim.x + blk] = mkc(re, im);
  }
}

// w[r] -= sum_v V_v[r] h[v*R + r].  A CTA of 256 threads covers SUB_ROWS =
// 128 rows; the two halves of the CTA take the two halves of the basis for
// the same rows (twice the loads in flight of one thread per row), 8 basis
// vectors in flight each, and are combined in shared memory in a fixed
// order.  Also writes the CTA's share of ||w[r]||^2 after the update to
// pnorm[r * gridDim.x + blockIdx.x] (FP64, reduced in a fixed order), zero
// for a right-hand side that is not active.
constexpr int SUB_ROWS = 128;
__global__ void __launch_bounds__(2 * SUB_ROWS) k_subtract_ff(const float4* __restrict__ V, int64_t vstride, int nvec,
                                                              const cd* __restrict__ h, float4* __restrict__ w, int R,
                                                              int64_t N, const int* __restrict__ active,
                                                              cd* __restrict__ pnorm) {
  const int r = blockIdx.y;
  if (!active[r]) {
    if (threadIdx.x == 0) pnorm[(int64_t)r * gridDim.x + blockIdx.x] = mkc(0.0, 0.0);
    return;
  }
  __shared__ float4 hs[MAX_RESTART + 1];
  __shared__ float4 other[SUB_ROWS];
  __shared__ double red[2 * SUB_ROWS / 32];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    const cd hv = h[v * R + r];
    hs[v] = split_ff(mkc(-hv.x, -hv.y));
  }
  const int row = threadIdx.x & (SUB_ROWS - 1), half = threadIdx.x / SUB_ROWS;
  const int nh = (nvec + 1) / 2;
  const int vb = half ? nh : 0, ve = half ? nvec : nh;
  __syncthreads();
  float4* wr = w + (int64_t)r * N;
  const float4* Vr = V + (int64_t)r * N;
  double acc = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * SUB_ROWS; base < N; base += (int64_t)gridDim.x * SUB_ROWS) {
    const int64_t i = base + row;
    const bool ok = i < N;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (ok) {
      if (!half) {
        const float4 w0 = wr[i];
        rh = w0.x;
        rl = w0.y;
        ih = w0.z;
        il = w0.w;
      }
      int v = vb;
      for (; v + 7 < ve; v += 8) {
        float4 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = Vr[(int64_t)(v + q) * vstride + i];
#pragma unroll
        for (int q = 0; q < 8; ++q) ff_cmac(a[q], hs[v + q], rh, rl, ih, il);
      }
      for (; v < ve; ++v) ff_cmac(Vr[(int64_t)v * vstride + i], hs[v], rh, rl, ih, il);
    }
    if (half) other[row] = make_float4(rh, rl, ih, il);
    __syncthreads();
    if (!half && ok) {
      const float4 o = other[row];
      float s1, e1, s2, e2;
      two_sum_f(rh, o.x, s1, e1);
      two_sum_f(ih, o.z, s2, e2);
      const float4 out = ff_norm(s1, (rl + o.y) + e1, s2, (il + o.w) + e2);
      wr[i] = out;
      const double re = (double)out.x + (double)out.y, im = (double)out.z + (double)out.w;
      acc = fma(re, re, fma(im, im, acc));
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < 2 * SUB_ROWS / 32; ++u) t += red[u];
    pnorm[(int64_t)r * gridDim.x + blockIdx.x] = mkc(t, 0.0);
  }
}

// Warp-parallel fixed-order sum of the nblk norm partials of rhs r.
__device__ __forceinline__ double warp_norm_sum(const cd* __restrict__ pnorm, int nblk, int r, int lane) {
  double t = 0.0;
  for (int b = lane; b < nblk; b += 32) t += pnorm[(int64_t)r * nblk + b].x;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// After the first Gram-Schmidt pass, one warp per rhs: ||w'||^2 from the
// subtract's partials, and need[r] = 1 when the pass removed more than half
// of ||w||^2 (before = ||w||^2 from the projection dots).
__global__ void k_norm_flag(const cd* __restrict__ pnorm, int nblk, const cd* __restrict__ before,
                            const int* __restrict__ active, cd* __restrict__ after, int* __restrict__ need, int R) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  const double a = warp_norm_sum(pnorm, nblk, r, lane);
  if (lane == 0) {
    after[r] = mkc(a, 0.0);
    need[r] = (active[r] && a < 0.5 * before[r].x) ? 1 : 0;
  }
}

// End of the Gram-Schmidt step, one warp per rhs: where the second pass ran,
// h += h2 and ||w||^2 from its partials; then ||w|| and 1 / ||w||.
__global__ void k_finish(const cd* __restrict__ pnorm, int nblk, const cd* __restrict__ first,
                         const int* __restrict__ need, const cd* __restrict__ h2, cd* __restrict__ h, int nvec,
                         double* __restrict__ wnorm, double* __restrict__ inv, int R) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  double w2 = first[r].x;
  if (need[r]) {
    w2 = warp_norm_sum(pnorm, nblk, r, lane);
    for (int v = lane; v < nvec; v += 32) h[v * R + r] = cadd(h[v * R + r], h2[v * R + r]);
  }
  if (lane == 0) {
    const double v = sqrt(fmax(w2, 0.0));
    wnorm[r] = v;
    inv[r] = v > 0.0 ? 1.0 / v : 0.0;
  }
}

// ------------------------------------- delayed reorthogonalisation (DCGS2) --
// Classical Gram-Schmidt with the second (reorthogonalising) pass of step
// j - 1 folded into the projections of step j, so that a step reads the basis
// twice instead of four times.  State at step j: q_0..q_{j-1} orthonormal in
// slots 0..j-1, the pending vector p (the product of step j - 1 projected
// once, not normalised) in slot j, and the first-pass coefficients s_prev of
// column j - 1.  With z = A p in slot j + 1:
//   t = Q^H p, b = Q^H z, pp = p^H p, pz = p^H z           (one dots pass)
//   beta = sqrt(pp - |t|^2),  q_j = (p - Q t) / beta
//   column j - 1 of H: s_prev + t, subdiagonal beta
//   c = [b ; (pz - t^H b) / beta] = Q_{j+1}^H z
//   next pending (z - Q_{j+1} c) / beta,  its first-pass coefficients
//   s = (c - H t) / beta  (H: the raw Hessenberg columns 0..j-1)
// (A q_j = (z - A Q t) / beta and A Q = Q_{j+1} H.)

// partial sums of conj(V_v) p and conj(V_v) z (v < nvec), DOT2_VB vectors per
// CTA, both targets from each loaded basis row (two vectors per CTA keep the
// registers low enough for four CTAs per SM)
constexpr int DOT2_VB = 2;
__global__ void __launch_bounds__(RED_THREADS) k_dots2_ff(const float4* __restrict__ V, int64_t vstride, int nvec,
                                                          const float4* __restrict__ p, const float4* __restrict__ z,
                                                          int R, int64_t N, cd* __restrict__ part_p,
                                                          cd* __restrict__ part_z, const int* __restrict__ active) {
  const int blk = blockIdx.x, v0 = blockIdx.y * DOT2_VB, r = blockIdx.z;
  const int nq = min(DOT2_VB, nvec - v0);
  float ph[DOT2_VB], pl[DOT2_VB], pih[DOT2_VB], pil[DOT2_VB];
  float zh[DOT2_VB], zl[DOT2_VB], zih[DOT2_VB], zil[DOT2_VB];
#pragma unroll
  for (int q = 0; q < DOT2_VB; ++q) ph[q] = pl[q] = pih[q] = pil[q] = zh[q] = zl[q] = zih[q] = zil[q] = 0.f;
  if (active[r]) {
    const float4* a = V + (int64_t)v0 * vstride + (int64_t)r * N;
    const float4* pr = p + (int64_t)r * N;
    const float4* zr = z + (int64_t)r * N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < N; i += stride) {
      const float4 yp = pr[i], yz = zr[i];
      float4 x[DOT2_VB];
#pragma unroll
      for (int q = 0; q < DOT2_VB; ++q) x[q] = q < nq ? a[(int64_t)q * vstride + i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < DOT2_VB; ++q) {
        const float4 cx = ff_conj(x[q]);
        ff_cmac(cx, yp, ph[q], pl[q], pih[q], pil[q]);
        ff_cmac(cx, yz, zh[q], zl[q], zih[q], zil[q]);
      }
    }
  }
  __shared__ float4 sh[2][RED_THREADS / 32][DOT2_VB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < DOT2_VB; ++q) {
    ff_warp_sum(ph[q], pl[q]);
    ff_warp_sum(pih[q], pil[q]);
    ff_warp_sum(zh[q], zl[q]);
    ff_warp_sum(zih[q], zil[q]);
    if (lane == 0) {
      sh[0][warp][q] = make_float4(ph[q], pl[q], pih[q], pil[q]);
      sh[1][warp][q] = make_float4(zh[q], zl[q], zih[q], zil[q]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * nq) {
    const int tgt = threadIdx.x / nq, q = threadIdx.x - tgt * nq;
    double re = 0.0, im = 0.0;
    for (int u = 0; u < RED_THREADS / 32; ++u) {
      const float4 t = sh[tgt][u][q];
      re += (double)t.x + (double)t.y;
      im += (double)t.z + (double)t.w;
    }
    cd* out = tgt ? part_z : part_p;
    out[((int64_t)(v0 + q) * R + r) * gridDim.x + blk] = mkc(re, im);
  }
}

// One CTA per rhs: beta, the final column j - 1 (hc, raw copy in Hraw,
// subdiagonal in wnorm) and the update coefficients c.  t = hA[0..j-1],
// pp = hA[j], b = hB[0..j-1], pz = hB[j].
// With part_p (and part_z) given, the CTA's threads first reduce the system's
// projection partials into hA[0..j+1] and hB[0..j], one entry per thread,
// each summed over its nblk row blocks in the fixed order of
// k_reduce_partials (loads issued eight at a time, so that a long basis does
// not wait on one L2 round trip per partial); then its first warp does the
// rest.  Stopped systems are left out, and nothing downstream reads their
// entries.
constexpr int COEF_THREADS = 256;
__global__ void __launch_bounds__(COEF_THREADS) k_dcgs_coef(GmresState s, cd* __restrict__ hA, cd* __restrict__ hB,
                                                             const cd* __restrict__ sprev, cd* __restrict__ hc,
                                                             cd* __restrict__ cbuf, cd* __restrict__ Hraw,
                                                             double* __restrict__ wnorm, int R, int m, int j,
                                                             const cd* __restrict__ part_p = nullptr,
                                                             const cd* __restrict__ part_z = nullptr, int nblk = 0) {
  const int r = blockIdx.x, lane = threadIdx.x & 31;
  if (!s.active[r]) return;   // uniform over the CTA
  if (part_p) {
    const int na = j + 2;
    for (int it = threadIdx.x; it < na + j + 1; it += blockDim.x) {
      const bool isz = it >= na;
      const int64_t e = (int64_t)(isz ? it - na : it) * R + r;
      const cd* src = (isz ? part_z : part_p) + e * nblk;
      cd a = mkc(0.0, 0.0);
      for (int b = 0; b < nblk; b += 8) {
        cd x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = b + u < nblk ? src[b + u] : mkc(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (b + u < nblk) a = cadd(a, x[u]);
      }
      (isz ? hB : hA)[e] = a;
    }
    __syncthreads();
  }
  if (threadIdx.x >= 32) return;
  double tt = 0.0, tbr = 0.0, tbi = 0.0;
  for (int v = lane; v < j; v += 32) {
    const cd t = hA[v * R + r], b = hB[v * R + r];
    tt = fma(t.x, t.x, fma(t.y, t.y, tt));
    tbr = fma(t.x, b.x, fma(t.y, b.y, tbr));   // conj(t) b
    tbi = fma(t.x, b.y, fma(-t.y, b.x, tbi));
  }
  for (int o = 16; o > 0; o >>= 1) {
    tt += __shfl_xor_sync(0xffffffffu, tt, o);
    tbr += __shfl_xor_sync(0xffffffffu, tbr, o);
    tbi += __shfl_xor_sync(0xffffffffu, tbi, o);
  }
  const double b2 = hA[j * R + r].x - tt;
  const double beta = b2 > 0.0 ? sqrt(b2) : 0.0;
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  cd* Hc = Hraw + ((int64_t)r * m + (j > 0 ? j - 1 : 0)) * (m + 1);
  for (int v = lane; v < j; v += 32) {
    const cd val = cadd(sprev[v * R + r], hA[v * R + r]);
    hc[v * R + r] = val;
    Hc[v] = val;
    cbuf[v * R + r] = hB[v * R + r];
  }
  if (lane == 0) {
    if (j > 0) {
      Hc[j] = mkc(beta, 0.0);
      wnorm[r] = beta;
    }
    const cd pz = hB[j * R + r];
    cbuf[j * R + r] = cmulr(mkc(pz.x - tbr, pz.y - tbi), inv);
    s.inv[r] = inv;
  }
}

// s_new[i] = (c_i - sum_{v < j} H[i][v] t_v) / beta for rows i <= j (the
// first-pass coefficients of the new pending column), one warp per row.
__global__ void k_hess_t(const int* __restrict__ active, const cd* __restrict__ Hraw, const cd* __restrict__ hA,
                         const cd* __restrict__ cbuf, const double* __restrict__ inv, cd* __restrict__ sprev, int R,
                         int m, int j) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int r = blockIdx.y;
  if (i > j || !active[r]) return;
  double gr = 0.0, gi = 0.0;
  for (int v = max(0, i - 1) + lane; v < j; v += 32) {
    const cd hv = Hraw[((int64_t)r * m + v) * (m + 1) + i], t = hA[v * R + r];
    gr = fma(hv.x, t.x, fma(-hv.y, t.y, gr));
    gi = fma(hv.x, t.y, fma(hv.y, t.x, gi));
  }
  for (int o = 16; o > 0; o >>= 1) {
    gr += __shfl_xor_sync(0xffffffffu, gr, o);
    gi += __shfl_xor_sync(0xffffffffu, gi, o);
  }
  if (lane == 0) {
    const cd c = cbuf[i * R + r];
    sprev[i * R + r] = cmulr(mkc(c.x - gr, c.y - gi), inv[r]);
  }
}

// q_j = (p - Q t) / beta into slot j and the next pending vector
// (z - Q c_{0..j-1} - q_j c_j) / beta into slot j + 1, in one pass over
// q_0..q_{j-1} (two products per loaded basis row).  The two halves of a CTA
// take the two halves of the basis for the same rows and are combined in
// shared memory in a fixed order.
__global__ void __launch_bounds__(2 * SUB_ROWS) k_update2_ff(float4* __restrict__ V, int64_t vstride, int j,
                                                             const cd* __restrict__ hA, const cd* __restrict__ cbuf,
                                                             const double* __restrict__ inv, int R, int64_t N,
                                                             const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  __shared__ float4 ts[MAX_RESTART], cs[MAX_RESTART];
  __shared__ float4 op[SUB_ROWS], oz[SUB_ROWS];
  for (int v = threadIdx.x; v < j; v += blockDim.x) {
    const cd t = hA[v * R + r], c = cbuf[v * R + r];
    ts[v] = split_ff(mkc(-t.x, -t.y));
    cs[v] = split_ff(mkc(-c.x, -c.y));
  }
  const ff invf = ff_from_d(inv[r]);
  const cd cj = cbuf[j * R + r];
  const float4 mcj = split_ff(mkc(-cj.x, -cj.y));
  const int row = threadIdx.x & (SUB_ROWS - 1), half = threadIdx.x / SUB_ROWS;
  const int nh = (j + 1) / 2;
  const int vb = half ? nh : 0, ve = half ? j : nh;
  __syncthreads();
  float4* P = V + (int64_t)j * vstride + (int64_t)r * N;
  float4* Z = V + (int64_t)(j + 1) * vstride + (int64_t)r * N;
  const float4* Vr = V + (int64_t)r * N;
  for (int64_t base = (int64_t)blockIdx.x * SUB_ROWS; base < N; base += (int64_t)gridDim.x * SUB_ROWS) {
    const int64_t i = base + row;
    const bool ok = i < N;
    float ph = 0.f, pl = 0.f, pih = 0.f, pil = 0.f, zh = 0.f, zl = 0.f, zih = 0.f, zil = 0.f;
    if (ok) {
      if (!half) {
        const float4 p0 = P[i], z0 = Z[i];
        ph = p0.x;
        pl = p0.y;
        pih = p0.z;
        pil = p0.w;
        zh = z0.x;
        zl = z0.y;
        zih = z0.z;
        zil = z0.w;
      }
      int v = vb;
      for (; v + 3 < ve; v += 4) {
        float4 a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Vr[(int64_t)(v + q) * vstride + i];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ff_cmac(a[q], ts[v + q], ph, pl, pih, pil);
          ff_cmac(a[q], cs[v + q], zh, zl, zih, zil);
        }
      }
      for (; v < ve; ++v) {
        const float4 a = Vr[(int64_t)v * vstride + i];
        ff_cmac(a, ts[v], ph, pl, pih, pil);
        ff_cmac(a, cs[v], zh, zl, zih, zil);
      }
    }
    if (half) {
      op[row] = make_float4(ph, pl, pih, pil);
      oz[row] = make_float4(zh, zl, zih, zil);
    }
    __syncthreads();
    if (!half && ok) {
      float s1, e1, s2, e2;
      const float4 a = op[row], b = oz[row];
      two_sum_f(ph, a.x, s1, e1);
      two_sum_f(pih, a.z, s2, e2);
      const float4 pv = ff_norm(s1, (pl + a.y) + e1, s2, (pil + a.w) + e2);
      const ff qre = ff_mul(ff{pv.x, pv.y}, invf), qim = ff_mul(ff{pv.z, pv.w}, invf);
      const float4 q = make_float4(qre.h, qre.l, qim.h, qim.l);
      two_sum_f(zh, b.x, s1, e1);
      two_sum_f(zih, b.z, s2, e2);
      float wh = s1, wl = (zl + b.y) + e1, wih = s2, wil = (zil + b.w) + e2;
      ff_cmac(q, mcj, wh, wl, wih, wil);
      const float4 wv = ff_norm(wh, wl, wih, wil);
      const ff wre = ff_mul(ff{wv.x, wv.y}, invf), wim = ff_mul(ff{wv.z, wv.w}, invf);
      P[i] = q;
      Z[i] = make_float4(wre.h, wre.l, wim.h, wim.l);
    }
    __syncthreads();
  }
}

// v[r] *= s[r] in float-float
__global__ void k_scale_ff(float4* __restrict__ v, const double* __restrict__ s, int R, int64_t N,
                           const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  const ff f = ff_from_d(s[r]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = v[(int64_t)r * N + i];
    const ff re = ff_mul(ff{a.x, a.y}, f), im = ff_mul(ff{a.z, a.w}, f);
    v[(int64_t)r * N + i] = make_float4(re.h, re.l, im.h, im.l);
  }
}

// y[r] = float-float(x[r] * s[r])
__global__ void k_scale_to_ff(const cd* __restrict__ x, float4* __restrict__ y, const double* __restrict__ s, int R,
                              int64_t N, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  const double f = s[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[(int64_t)r * N + i] = split_ff(cmulr(x[(int64_t)r * N + i], f));
}

__global__ void k_cd_to_ff(const cd* __restrict__ x, float4* __restrict__ y, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = split_ff(x[i]);
}

__global__ void k_ff_to_cd(const float4* __restrict__ x, cd* __restrict__ y, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = ff_to_cd(x[i]);
}

// x[r] += sum_{i < jcount[r]} V_i[r] y_i[r]  (FP64 accumulation)
__global__ void k_update_x_ff(const float4* __restrict__ V, int64_t vstride, GmresState s, cd* __restrict__ x, int R,
                              int m, int64_t N) {
  const int r = blockIdx.y;
  const int J = s.jcount[r];
  if (J == 0) return;
  const cd* y = s.g + r * (m + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    cd acc = x[(int64_t)r * N + i];
    for (int v = 0; v < J; ++v) acc = cfma(ff_to_cd(V[(int64_t)v * vstride + (int64_t)r * N + i]), y[v], acc);
    x[(int64_t)r * N + i] = acc;
  }
}

// ---------------------------------------------------- FP32 Krylov basis --
// Operators whose products carry BF16 rounding (BF16 tensor-core operators
// and the inner solves of GMRES-IR) keep their basis in complex FP32: every
// Gram-Schmidt pass moves half the bytes of a float-float basis and needs a
// small fraction of its instructions.  The per-thread FP32 sums (a few
// thousand terms at most, relative error far below the BF16 rounding of the
// products) are reduced across threads in FP64, and the coefficients, the
// Hessenberg matrix and the rotations stay FP64 as in the float-float path.

__device__ __forceinline__ void cmac_conj_f(float2 x, float2 y, float& re, float& im) {   // += conj(x) y
  re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
  im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
}
__device__ __forceinline__ void cmac_f(float2 a, float2 b, float& re, float& im) {   // += a b
  re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
  im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
}
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 basis: partial sums of conj(V_v) p and (if z) conj(V_v) z for v < nvec,
// DOTF_VB vectors per CTA; per-thread FP32 sums, FP64 across threads in a
// fixed order.  Same partial layout as k_dots2_ff.
constexpr int DOTF_VB = 8;
// Grid extent over systems of the FP32-basis kernels, which loop over the rest.
constexpr int SYS_GRID = 64;
__global__ void __launch_bounds__(RED_THREADS) k_dots2_f32(const float2* __restrict__ V, int64_t vstride, int nvec,
                                                           const float2* __restrict__ p, const float2* __restrict__ z,
                                                           int R, int64_t N, cd* __restrict__ part_p,
                                                           cd* __restrict__ part_z, const int* __restrict__ active) {
  const int blk = blockIdx.x, v0 = blockIdx.y * DOTF_VB;
  const int nq = min(DOTF_VB, nvec - v0);
  const int ntgt = z ? 2 : 1;
  __shared__ cd sh[2][RED_THREADS / 32][DOTF_VB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // systems r = blockIdx.z, + gridDim.z, ...: a batch of many systems, most
  // of them stopped, costs no CTA launches for the stopped ones
  for (int r = blockIdx.z; r < R; r += gridDim.z) {
    if (!active[r]) {
      if (threadIdx.x < ntgt * nq) {
        const int tgt = threadIdx.x / nq, q = threadIdx.x - tgt * nq;
        (tgt ? part_z : part_p)[((int64_t)(v0 + q) * R + r) * gridDim.x + blk] = mkc(0.0, 0.0);
      }
      continue;
    }
    float pr[DOTF_VB], pi[DOTF_VB], zr[DOTF_VB], zi[DOTF_VB];
#pragma unroll
    for (int q = 0; q < DOTF_VB; ++q) pr[q] = pi[q] = zr[q] = zi[q] = 0.f;
    const float2* a = V + (int64_t)v0 * vstride + (int64_t)r * N;
    const float2* pp = p + (int64_t)r * N;
    const float2* zz = z ? z + (int64_t)r * N : nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < N; i += stride) {
      const float2 yp = pp[i];
      const float2 yz = zz ? zz[i] : make_float2(0.f, 0.f);
      float2 x[DOTF_VB];
#pragma unroll
      for (int q = 0; q < DOTF_VB; ++q) x[q] = q < nq ? a[(int64_t)q * vstride + i] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < DOTF_VB; ++q) {
        cmac_conj_f(x[q], yp, pr[q], pi[q]);
        cmac_conj_f(x[q], yz, zr[q], zi[q]);
      }
    }
    __syncthreads();   // the previous system's reads of sh are done
#pragma unroll
    for (int q = 0; q < DOTF_VB; ++q) {
      const double a0 = warp_sum_d((double)pr[q]), b0 = warp_sum_d((double)pi[q]);
      const double c0 = warp_sum_d((double)zr[q]), d0 = warp_sum_d((double)zi[q]);
      if (lane == 0) {
        sh[0][warp][q] = mkc(a0, b0);
        sh[1][warp][q] = mkc(c0, d0);
      }
    }
    __syncthreads();
    if (threadIdx.x < ntgt * nq) {
      const int tgt = threadIdx.x / nq, q = threadIdx.x - tgt * nq;
      double re = 0.0, im = 0.0;
      for (int u = 0; u < RED_THREADS / 32; ++u) {
        re += sh[tgt][u][q].x;
        im += sh[tgt][u][q].y;
      }
      (tgt ? part_z : part_p)[((int64_t)(v0 + q) * R + r) * gridDim.x + blk] = mkc(re, im);
    }
  }
}

// FP32 basis: q_j = (p - Q t) / beta into slot j and the next pending vector
// (z - Q c_{0..j-1} - q_j c_j) / beta into slot j + 1 (the step of
// k_update2_ff), the two halves of a CTA taking the two halves of the basis.
__global__ void __launch_bounds__(2 * SUB_ROWS) k_update2_f32(float2* __restrict__ V, int64_t vstride, int j,
                                                              const cd* __restrict__ hA, const cd* __restrict__ cbuf,
                                                              const double* __restrict__ inv, int R, int64_t N,
                                                              const int* __restrict__ active) {
  __shared__ float2 ts[MAX_RESTART], cs[MAX_RESTART];
  __shared__ float2 op[SUB_ROWS], oz[SUB_ROWS];
  // systems r = blockIdx.y, + gridDim.y, ... (stopped systems cost no CTA launches)
  for (int r = blockIdx.y; r < R; r += gridDim.y) {
    if (!active[r]) continue;
    __syncthreads();   // the previous system's reads of ts, cs are done
    for (int v = threadIdx.x; v < j; v += blockDim.x) {
      const cd t = hA[v * R + r], c = cbuf[v * R + r];
      ts[v] = make_float2((float)-t.x, (float)-t.y);
      cs[v] = make_float2((float)-c.x, (float)-c.y);
    }
    const float invf = (float)inv[r];
    const cd cj = cbuf[j * R + r];
    const float2 mcj = make_float2((float)-cj.x, (float)-cj.y);
    const int row = threadIdx.x & (SUB_ROWS - 1), half = threadIdx.x / SUB_ROWS;
    const int nh = (j + 1) / 2;
    const int vb = half ? nh : 0, ve = half ? j : nh;
    __syncthreads();
    float2* P = V + (int64_t)j * vstride + (int64_t)r * N;
    float2* Z = V + (int64_t)(j + 1) * vstride + (int64_t)r * N;
    const float2* Vr = V + (int64_t)r * N;
    for (int64_t base = (int64_t)blockIdx.x * SUB_ROWS; base < N; base += (int64_t)gridDim.x * SUB_ROWS) {
      const int64_t i = base + row;
      const bool ok = i < N;
      float pre = 0.f, pim = 0.f, zre = 0.f, zim = 0.f;
      if (ok) {
        if (!half) {
          const float2 p0 = P[i], z0 = Z[i];
          pre = p0.x;
          pim = p0.y;
          zre = z0.x;
          zim = z0.y;
        }
        int v = vb;
        for (; v + 3 < ve; v += 4) {
          float2 a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = Vr[(int64_t)(v + q) * vstride + i];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            cmac_f(a[q], ts[v + q], pre, pim);
            cmac_f(a[q], cs[v + q], zre, zim);
          }
        }
        for (; v < ve; ++v) {
          const float2 a = Vr[(int64_t)v * vstride + i];
          cmac_f(a, ts[v], pre, pim);
          cmac_f(a, cs[v], zre, zim);
        }
      }
      if (half) {
        op[row] = make_float2(pre, pim);
        oz[row] = make_float2(zre, zim);
      }
      __syncthreads();
      if (!half && ok) {
        const float2 a = op[row], b = oz[row];
        const float2 q = make_float2((pre + a.x) * invf, (pim + a.y) * invf);
        float wre = zre + b.x, wim = zim + b.y;
        cmac_f(q, mcj, wre, wim);
        P[i] = q;
        Z[i] = make_float2(wre * invf, wim * invf);
      }
      __syncthreads();
    }
  }
}

// y[r] = FP32(x[r] * s[r])
__global__ void k_scale_to_f32(const cd* __restrict__ x, float2* __restrict__ y, const double* __restrict__ s, int R,
                               int64_t N, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  const double f = s[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const cd v = x[(int64_t)r * N + i];
    y[(int64_t)r * N + i] = make_float2((float)(v.x * f), (float)(v.y * f));
  }
}

// x[r] += sum_{i < jcount[r]} V_i[r] y_i[r] with an FP32 basis: the
// correction is summed in FP32 (the basis and the products behind it carry
// far larger roundings) and added to x in FP64.
__global__ void k_update_x_f32(const float2* __restrict__ V, int64_t vstride, GmresState s, cd* __restrict__ x, int R,
                               int m, int64_t N) {
  const int r = blockIdx.y;
  const int J = s.jcount[r];
  if (J == 0) return;
  __shared__ float2 ys[MAX_RESTART];
  for (int v = threadIdx.x; v < J; v += blockDim.x) {
    const cd y = s.g[r * (m + 1) + v];
    ys[v] = make_float2((float)y.x, (float)y.y);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int v = 0; v < J; ++v) cmac_f(V[(int64_t)v * vstride + (int64_t)r * N + i], ys[v], re, im);
    cd& xi = x[(int64_t)r * N + i];
    xi = mkc(xi.x + (double)re, xi.y + (double)im);
  }
}

// NaN / Inf scan of the right-hand side.
__global__ void k_finite_check(const cd* __restrict__ b, int64_t total, int* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = b[i];
    if (!isfinite(v.x) || !isfinite(v.y)) *bad = 1;
  }
}

// Iterations to enqueue before the host reads the convergence flags again:
// half of the iterations still needed at the residual contraction rate seen
// since the last look (1 to 32), so that a solve overshoots its convergence
// by a few iterations at most while most host round trips disappear.
static int next_block(double last, double cur, int since, double tol) {
  if (!(last > 0.0) || !(cur > 0.0) || since < 1) return 4;
  if (cur >= last) return 16;   // stagnating within the cycle
  const double rate = std::pow(cur / last, 1.0 / since);
  const double need = std::log(tol / cur) / std::log(rate);
  if (!(need > 0.0)) return 1;
  return (int)std::max(1.0, std::min(32.0, std::floor(0.5 * need)));
}

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

fmpb_status gmres_solve(const MatvecFn& A, int R, int64_t N, const cd* b, cd* x, const fmpb_solve_opts& o,
                        fmpb_solve_info* info, cudaStream_t st, const MatvecFfFn* Aff, int* active_host,
                        const MatvecF32Fn* A32) {
  const double tol = o.tol > 0 ? o.tol : 1e-8;
  const int m = o.restart > 0 ? o.restart : 30;
  const int maxit = o.maxit > 0 ? o.maxit : 1000;
  if (m > MAX_RESTART || R < 1 || N < 1) {
    set_error("gmres: restart must be 1..%d and R, N positive", MAX_RESTART);
    return FMPB_EINVAL;
  }
  auto t0 = std::chrono::steady_clock::now();
  const int64_t vstride = (int64_t)R * N;
  const bool f32b = A32 != nullptr;   // FP32 Krylov basis (float2 values)
  const size_t vbytes = f32b ? sizeof(float2) : sizeof(float4);
  // device memory: basis (m+1) R N, work vector R N, small state
  DevBuf Vb, Wb, Tb, Sb, Pb;
  // control state: carve one allocation; the first pass (base = null) sizes it
  GmresState s;
  cd *h = nullptr, *h2 = nullptr, *nrm2 = nullptr, *pnorm = nullptr;
  cd *hB = nullptr, *sprev = nullptr, *cbuf = nullptr, *hc = nullptr;
  double *wnorm = nullptr;
  int *all_active = nullptr, *bad = nullptr, *need = nullptr;
  size_t small = 0;
  for (int pass = 0; pass < 2; ++pass) {
    char* base = (char*)Sb.p;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
      void* p = base ? (void*)(base + off) : nullptr;
      off += (bytes + 255) / 256 * 256;
      return p;
    };
    s.H = (cd*)take(sizeof(cd) * (size_t)R * (m + 1) * m);
    s.sn = (cd*)take(sizeof(cd) * (size_t)R * m);
    s.g = (cd*)take(sizeof(cd) * (size_t)R * (m + 1));
    h = (cd*)take(sizeof(cd) * (size_t)R * (m + 2));
    h2 = (cd*)take(sizeof(cd) * (size_t)R * (m + 1));
    nrm2 = (cd*)take(sizeof(cd) * 2 * (size_t)R);
    hB = (cd*)take(sizeof(cd) * (size_t)R * (m + 2));
    sprev = (cd*)take(sizeof(cd) * (size_t)R * (m + 1));
    cbuf = (cd*)take(sizeof(cd) * (size_t)R * (m + 1));
    hc = (cd*)take(sizeof(cd) * (size_t)R * (m + 1));
    pnorm = (cd*)take(sizeof(cd) * (size_t)R * 152 * 8);
    s.cs = (double*)take(sizeof(double) * (size_t)R * m);
    s.beta = (double*)take(sizeof(double) * R);
    s.inv = (double*)take(sizeof(double) * R);
    s.bnorm = (double*)take(sizeof(double) * R);
    s.resid = (double*)take(sizeof(double) * R);
    wnorm = (double*)take(sizeof(double) * R);
    s.active = (int*)take(sizeof(int) * R);
    s.jcount = (int*)take(sizeof(int) * R);
    s.iters = (int*)take(sizeof(int) * R);
    all_active = (int*)take(sizeof(int) * R);
    need = (int*)take(sizeof(int) * R);
    bad = (int*)take(sizeof(int));
    if (pass == 0) {
      small = off;
      if (cudaMalloc(&Vb.p, vbytes * (size_t)(m + 1) * vstride) != cudaSuccess ||
          cudaMalloc(&Wb.p, sizeof(cd) * (size_t)vstride) != cudaSuccess ||
          cudaMalloc(&Tb.p, sizeof(cd) * (size_t)vstride) != cudaSuccess || cudaMalloc(&Sb.p, small) != cudaSuccess ||
          cudaMalloc(&Pb.p, 2 * sizeof(cd) * (size_t)(m + 2) * R * RED_BLOCKS) != cudaSuccess) {
        cudaGetLastError();
        set_error("gmres: cannot allocate the Krylov basis (%zu bytes)", sizeof(cd) * (size_t)(m + 2) * vstride);
        return FMPB_ENOMEM;
      }
    }
  }
  float4* V = (float4*)Vb.p;   // float-float basis
  float2* V32 = (float2*)Vb.p;  // or the FP32 basis
  cd* W = (cd*)Wb.p;           // product output / residual (FP64)
  cd* T = (cd*)Tb.p;           // product input (FP64 copy of v_j)
  cd* partial = (cd*)Pb.p;
  cd* partial2 = partial + (size_t)(m + 2) * R * RED_BLOCKS;
  // delayed reorthogonalisation (one basis read less per pass) where the
  // operator multiplies float-float vectors, with the raw Hessenberg columns
  // kept for the H t corrections
  DevBuf Hb;
  const size_t hraw_bytes = sizeof(cd) * (size_t)R * m * (m + 1);
  const bool dcgs2 = (Aff != nullptr || f32b) && hraw_bytes <= ((size_t)1 << 30) &&
                     cudaMalloc(&Hb.p, hraw_bytes) == cudaSuccess;
  if (!dcgs2) cudaGetLastError();
  if (f32b && !dcgs2) {
    set_error("gmres: cannot allocate the Hessenberg copy (%zu bytes) of the FP32-basis solver", hraw_bytes);
    return FMPB_ENOMEM;
  }
  cd* Hraw = (cd*)Hb.p;

  const unsigned vec_blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 152 * 4);
  const unsigned sub_blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + SUB_ROWS - 1) / SUB_ROWS, 152 * 8));
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, N / (RED_THREADS * 8)));
  const unsigned rb = grid_for(R, 64);

  // all-active mask for norms of b and of true residuals
  std::vector<int> ones(R, 1);
  FMPB_CUDA(cudaMemcpyAsync(all_active, ones.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
  FMPB_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  FMPB_LAUNCH("finite_check", st, k_finite_check<<<vec_blocks, 256, 0, st>>>(b, vstride, bad));
  int hbad = 0;
  FMPB_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaStreamSynchronize(st));
  if (hbad) {
    set_error("gmres: the right-hand side holds NaN or Inf");
    return FMPB_ENAN;
  }

  auto norms = [&](const cd* X, double* out, double* invout) -> fmpb_status {
    FMPB_LAUNCH("dots", st, k_dots<<<dim3(nb, 1, R), RED_THREADS, 0, st>>>(X, 0, 1, X, R, N, partial, all_active));
    FMPB_LAUNCH("reduce_partials", st, k_reduce_partials<<<grid_for(R, 64), 64, 0, st>>>(partial, nb, R, nrm2, 0));
    FMPB_LAUNCH("sqrt_real", st, k_sqrt_real<<<rb, 64, 0, st>>>(nrm2, out, invout, R));
    FMPB_CUDA(cudaGetLastError());
    return FMPB_OK;
  };

  FMPB_TRY(norms(b, s.bnorm, nullptr));
  FMPB_CUDA(cudaMemsetAsync(x, 0, sizeof(cd) * vstride, st));
  FMPB_CUDA(cudaMemsetAsync(s.iters, 0, sizeof(int) * R, st));

  std::vector<double> hres(R), hbn(R), hest(R);
  std::vector<int> hact(R), iters(R, 0);
  auto publish = [&](bool all) {
    if (active_host)
      for (int r = 0; r < R; ++r) active_host[r] = all ? 1 : hact[r];
  };
  int total_it = 0;
  bool timed_out = false;
  bool first = true;
  while (true) {
    // r0 = b - A x  (x = 0 on the first cycle)
    publish(true);
    if (first) {
      FMPB_CUDA(cudaMemcpyAsync(W, b, sizeof(cd) * vstride, cudaMemcpyDeviceToDevice, st));
    } else {
      FMPB_TRY(A(R, x, W, st));
      FMPB_LAUNCH("residual", st, k_residual<<<vec_blocks, 256, 0, st>>>(b, W, vstride));
    }
    first = false;
    FMPB_TRY(norms(W, s.beta, s.inv));
    FMPB_LAUNCH("cycle_start", st, k_cycle_start<<<rb, 64, 0, st>>>(s, R, m, tol));
    if (f32b)
      FMPB_LAUNCH("scale_to_f32", st, k_scale_to_f32<<<dim3(vec_blocks, R), 256, 0, st>>>(W, V32, s.inv, R, N, s.active));
    else
      FMPB_LAUNCH("scale_to_ff", st, k_scale_to_ff<<<dim3(vec_blocks, R), 256, 0, st>>>(W, V, s.inv, R, N, s.active));
    FMPB_CUDA(cudaGetLastError());
    FMPB_CUDA(cudaMemcpyAsync(hact.data(), s.active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    FMPB_CUDA(cudaStreamSynchronize(st));
    publish(false);
    bool any = false;
    for (int r = 0; r < R; ++r) any |= hact[r] != 0;
    if (!any) break;
    int block = 4, since = 0;
    double last_res = -1.0;
    if (dcgs2) {
      int jdone = 0;
      for (int j = 0; j < m && total_it < maxit; ++j) {
        float4* vj = V + (int64_t)j * vstride;       // pending p
        float4* vn = V + (int64_t)(j + 1) * vstride; // z = A p
        float2* vj32 = V32 + (int64_t)j * vstride;
        float2* vn32 = V32 + (int64_t)(j + 1) * vstride;
        if (f32b)
          FMPB_TRY((*A32)(R, vj32, vn32, st));
        else
          FMPB_TRY((*Aff)(R, vj, vn, st));
        jdone = j + 1;
        // row blocks per vector group: about two waves of CTAs in total, so
        // that a long basis gives each thread many rows and the per-CTA
        // reduction is amortised (a short one keeps up to nb row blocks)
        const int vper = f32b ? DOTF_VB : DOT2_VB;
        const int vg = (j + 2 + vper - 1) / vper;
        const int Rg = f32b ? std::min(R, SYS_GRID) : R;   // FP32 kernels loop over systems
        const int nb2 = std::max(1, std::min(nb, (152 * 4 * 2 + vg * Rg - 1) / (vg * Rg)));
        if (f32b)
          FMPB_LAUNCH("dots_dcgs2_f32", st, k_dots2_f32<<<dim3(nb2, vg, Rg), RED_THREADS, 0, st>>>(V32, vstride, j + 2, vj32, vn32, R, N, partial, partial2, s.active));
        else
          FMPB_LAUNCH("dots_dcgs2", st, k_dots2_ff<<<dim3(nb2, vg, R), RED_THREADS, 0, st>>>(V, vstride, j + 2, vj, vn, R, N, partial, partial2, s.active));
        FMPB_LAUNCH("dcgs2_coef", st, k_dcgs_coef<<<R, COEF_THREADS, 0, st>>>(s, h, hB, sprev, hc, cbuf, Hraw, wnorm, R, m, j, partial, partial2, nb2));
        FMPB_LAUNCH("dcgs2_hess_t", st, k_hess_t<<<dim3((unsigned)((j + 1 + 7) / 8), R), 256, 0, st>>>(s.active, Hraw, h, cbuf, s.inv, sprev, R, m, j));
        if (f32b)
          FMPB_LAUNCH("update_dcgs2_f32", st, k_update2_f32<<<dim3(sub_blocks, std::min(R, SYS_GRID)), 256, 0, st>>>(V32, vstride, j, h, cbuf, s.inv, R, N, s.active));
        else
          FMPB_LAUNCH("update_dcgs2", st, k_update2_ff<<<dim3(sub_blocks, R), 256, 0, st>>>(V, vstride, j, h, cbuf, s.inv, R, N, s.active));
        if (j >= 1) FMPB_LAUNCH("givens", st, k_givens<<<R, 32 * GIV_WARPS, 0, st>>>(s, hc, wnorm, R, m, j - 1, tol));
        FMPB_CUDA(cudaGetLastError());
        ++total_it;
        // The host looks at the convergence flags only every `block`
        // iterations; in between it keeps enqueueing, and the Arnoldi kernels
        // of converged right-hand sides return at once (device-side flags).
        if (++since < block && j + 1 < m && total_it < maxit) continue;
        FMPB_CUDA(cudaMemcpyAsync(hact.data(), s.active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        FMPB_CUDA(cudaMemcpyAsync(hest.data(), s.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        FMPB_CUDA(cudaStreamSynchronize(st));
        publish(false);
        any = false;
        double cur = 0.0;
        for (int r = 0; r < R; ++r)
          if (hact[r]) {
            any = true;
            cur = std::max(cur, hest[r]);
          }
        if (!any) break;
        if (o.timeout_ms > 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
                o.timeout_ms) {
          timed_out = true;
          break;
        }
        block = next_block(last_res, cur, since, tol);
        last_res = cur;
        since = 0;
      }
      // finish the pending column (a full cycle, or the iteration limit)
      if (any && jdone > 0) {
        if (f32b)
          FMPB_LAUNCH("dots", st, k_dots2_f32<<<dim3(nb, (jdone + 1 + DOTF_VB - 1) / DOTF_VB, std::min(R, SYS_GRID)), RED_THREADS, 0, st>>>(V32, vstride, jdone + 1, V32 + (int64_t)jdone * vstride, nullptr, R, N, partial, nullptr, s.active));
        else
          FMPB_LAUNCH("dots", st, k_dots_ff4<<<dim3(nb, (jdone + 1 + DOT_VB - 1) / DOT_VB, R), RED_THREADS, 0, st>>>(V, vstride, jdone + 1, V + (int64_t)jdone * vstride, R, N, partial, s.active));
        FMPB_LAUNCH("reduce_partials", st, k_reduce_partials<<<grid_for((jdone + 1) * R, 64), 64, 0, st>>>(partial, nb, (jdone + 1) * R, h, 0));
        FMPB_LAUNCH("dcgs2_coef", st, k_dcgs_coef<<<R, COEF_THREADS, 0, st>>>(s, h, h, sprev, hc, cbuf, Hraw, wnorm, R, m, jdone));
        FMPB_LAUNCH("givens", st, k_givens<<<R, 32 * GIV_WARPS, 0, st>>>(s, hc, wnorm, R, m, jdone - 1, tol));
        FMPB_CUDA(cudaGetLastError());
      }
    } else {
      for (int j = 0; j < m && total_it < maxit; ++j) {
        float4* vj = V + (int64_t)j * vstride;
        float4* vn = V + (int64_t)(j + 1) * vstride;
        if (Aff) {
          FMPB_TRY((*Aff)(R, vj, vn, st));
        } else {
          FMPB_LAUNCH("ff_to_cd", st, k_ff_to_cd<<<vec_blocks, 256, 0, st>>>(vj, T, vstride));
          FMPB_TRY(A(R, T, W, st));
          FMPB_LAUNCH("cd_to_ff", st, k_cd_to_ff<<<vec_blocks, 256, 0, st>>>(W, vn, vstride));
        }
        // classical Gram-Schmidt against v_0..v_j, repeated when the first
        // pass lost more than half of ||w||^2.  w sits in slot j + 1 of the
        // basis, so one launch over slots 0..j+1 gives the projections h_0..h_j
        // and ||w||^2 (entry j + 1).
        FMPB_LAUNCH("dots", st, k_dots_ff4<<<dim3(nb, (j + 2 + DOT_VB - 1) / DOT_VB, R), RED_THREADS, 0, st>>>(V, vstride, j + 2, vn, R, N, partial, s.active));
        FMPB_LAUNCH("reduce_partials", st, k_reduce_partials<<<grid_for((j + 2) * R, 64), 64, 0, st>>>(partial, nb, (j + 2) * R, h, 0));
        FMPB_LAUNCH("subtract_projection", st, k_subtract_ff<<<dim3(sub_blocks, R), 256, 0, st>>>(V, vstride, j + 1, h, vn, R, N, s.active, pnorm));
        FMPB_LAUNCH("reorth_flag", st, k_norm_flag<<<grid_for(R, 4), 128, 0, st>>>(pnorm, (int)sub_blocks, h + (int64_t)(j + 1) * R, s.active, nrm2, need, R));
        FMPB_LAUNCH("dots_reorth", st, k_dots_ff4<<<dim3(nb, (j + 1 + DOT_VB - 1) / DOT_VB, R), RED_THREADS, 0, st>>>(V, vstride, j + 1, vn, R, N, partial, need));
        FMPB_LAUNCH("reduce_partials", st, k_reduce_partials<<<grid_for((j + 1) * R, 64), 64, 0, st>>>(partial, nb, (j + 1) * R, h2, 0));
        FMPB_LAUNCH("subtract_reorth", st, k_subtract_ff<<<dim3(sub_blocks, R), 256, 0, st>>>(V, vstride, j + 1, h2, vn, R, N, need, pnorm));
        // h += h2 and ||w|| where the second pass ran; normalise
        FMPB_LAUNCH("sqrt_real", st, k_finish<<<grid_for(R, 4), 128, 0, st>>>(pnorm, (int)sub_blocks, nrm2, need, h2, h, j + 1, wnorm, s.inv, R));
        FMPB_LAUNCH("scale", st, k_scale_ff<<<dim3(vec_blocks, R), 256, 0, st>>>(vn, s.inv, R, N, s.active));
        FMPB_LAUNCH("givens", st, k_givens<<<R, 32 * GIV_WARPS, 0, st>>>(s, h, wnorm, R, m, j, tol));
        FMPB_CUDA(cudaGetLastError());
        ++total_it;
        // The host looks at the convergence flags only every `block`
        // iterations; in between it keeps enqueueing, and the Arnoldi kernels
        // of converged right-hand sides return at once (device-side flags).
        if (++since < block && j + 1 < m && total_it < maxit) continue;
        FMPB_CUDA(cudaMemcpyAsync(hact.data(), s.active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        FMPB_CUDA(cudaMemcpyAsync(hest.data(), s.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        FMPB_CUDA(cudaStreamSynchronize(st));
        publish(false);
        any = false;
        double cur = 0.0;
        for (int r = 0; r < R; ++r)
          if (hact[r]) {
            any = true;
            cur = std::max(cur, hest[r]);
          }
        if (!any) break;
        if (o.timeout_ms > 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
                o.timeout_ms) {
          timed_out = true;
          break;
        }
        block = next_block(last_res, cur, since, tol);
        last_res = cur;
        since = 0;
      }
    }
    FMPB_LAUNCH("backsolve", st, k_backsolve<<<R, 32, 0, st>>>(s, R, m));
    if (f32b)
      FMPB_LAUNCH("update_x", st, k_update_x_f32<<<dim3(vec_blocks, R), 256, 0, st>>>(V32, vstride, s, x, R, m, N));
    else
      FMPB_LAUNCH("update_x", st, k_update_x_ff<<<dim3(vec_blocks, R), 256, 0, st>>>(V, vstride, s, x, R, m, N));
    FMPB_CUDA(cudaGetLastError());
    if (!any || timed_out || total_it >= maxit) break;
  }
  // true residual with one more product
  publish(true);
  FMPB_TRY(A(R, x, W, st));
  FMPB_LAUNCH("residual", st, k_residual<<<vec_blocks, 256, 0, st>>>(b, W, vstride));
  FMPB_TRY(norms(W, s.beta, nullptr));
  FMPB_CUDA(cudaMemcpyAsync(hres.data(), s.beta, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaMemcpyAsync(hbn.data(), s.bnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaMemcpyAsync(hest.data(), s.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaMemcpyAsync(iters.data(), s.iters, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaStreamSynchronize(st));
  bool all_conv = true;
  for (int r = 0; r < R; ++r) {
    double rel = hbn[r] > 0 ? hres[r] / hbn[r] : 0.0;
    bool conv = hest[r] <= tol;
    all_conv &= conv;
    if (info) {
      info[r].iters = iters[r];
      info[r].converged = conv ? 1 : 0;
      info[r].relres_est = hest[r];
      info[r].relres_true = rel;
      info[r].refinements = 0;
    }
  }
  if (timed_out) {
    set_error("gmres: wall-clock limit of %d ms reached", o.timeout_ms);
    return FMPB_ETIMEOUT;
  }
  if (!all_conv) {
    set_error("gmres: tolerance %.3g not reached within %d iterations", tol, maxit);
    return FMPB_ENOCONV;
  }
  return FMPB_OK;
}

}  // namespace fmpb

namespace fmpb {

// r = b - r for rhs not yet converged, r = 0 for converged ones
__global__ void k_outer_residual(const cd* __restrict__ b, cd* __restrict__ r, const int* __restrict__ done, int R,
                                 int64_t N, int from_product) {
  const int rr = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = (int64_t)rr * N + i;
    r[k] = done[rr] ? mkc(0.0, 0.0) : (from_product ? csub(b[k], r[k]) : b[k]);
  }
}

__global__ void k_axpy(cd* __restrict__ x, const cd* __restrict__ d, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = cadd(x[i], d[i]);
}

__global__ void k_norm2_partial(const cd* __restrict__ v, int64_t N, double* __restrict__ out) {
  const int r = blockIdx.y;
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const cd a = v[(int64_t)r * N + i];
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)r * gridDim.x + blockIdx.x] = sh[0];
}

// Mixed-precision iterative refinement (GMRES-IR): the residual
// r = b - A x is formed with the accurate operator, the correction equation
// A_low d = r is solved by GMRES with the low-precision operator to the
// relative tolerance inner_tol, and x += d, until ||r|| / ||b|| <= tol.
fmpb_status gmres_refined(const MatvecFn& A, const MatvecFn& Alow, int R, int64_t N, const cd* b, cd* x,
                          const fmpb_solve_opts& o, fmpb_solve_info* info, cudaStream_t st,
                          const MatvecF32Fn* Alow32) {
  const double tol = o.tol > 0 ? o.tol : 1e-8;
  const double inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-4;
  const int maxit = o.maxit > 0 ? o.maxit : 1000;
  const int64_t total = (int64_t)R * N;
  auto t0 = std::chrono::steady_clock::now();
  cd *r = nullptr, *d = nullptr;
  double* part = nullptr;
  int* done = nullptr;
  const unsigned nbk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 64));
  struct Free {
    void* p[4];
    ~Free() {
      for (void* q : p)
        if (q) cudaFree(q);
    }
  } fr{{nullptr, nullptr, nullptr, nullptr}};
  if (cudaMalloc(&r, sizeof(cd) * total) != cudaSuccess || cudaMalloc(&d, sizeof(cd) * total) != cudaSuccess ||
      cudaMalloc(&part, sizeof(double) * R * nbk) != cudaSuccess || cudaMalloc(&done, sizeof(int) * R) != cudaSuccess) {
    cudaGetLastError();
    set_error("gmres_refined: cannot allocate work vectors");
    return FMPB_ENOMEM;
  }
  fr.p[0] = r;
  fr.p[1] = d;
  fr.p[2] = part;
  fr.p[3] = done;
  const unsigned vb = (unsigned)std::min<int64_t>((N + 255) / 256, 152 * 4);
  std::vector<double> hp((size_t)R * nbk), bn(R), rn(R);
  std::vector<int> hdone(R, 0), iters(R, 0);
  auto norms = [&](const cd* v, std::vector<double>& out) -> fmpb_status {
    FMPB_LAUNCH("norm2", st, k_norm2_partial<<<dim3(nbk, R), 256, 0, st>>>(v, N, part));
    FMPB_CUDA(cudaGetLastError());
    FMPB_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * R * nbk, cudaMemcpyDeviceToHost, st));
    FMPB_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < R; ++q) {
      double s = 0.0;
      for (unsigned k = 0; k < nbk; ++k) s += hp[(size_t)q * nbk + k];
      out[q] = sqrt(s);
    }
    return FMPB_OK;
  };
  FMPB_TRY(norms(b, bn));
  for (int q = 0; q < R; ++q)
    if (!std::isfinite(bn[q])) {
      set_error("gmres_refined: the right-hand side holds NaN or Inf");
      return FMPB_ENAN;
    }
  FMPB_CUDA(cudaMemsetAsync(x, 0, sizeof(cd) * total, st));
  int refinements = 0, total_it = 0;
  std::vector<double> rel(R, 1.0);
  fmpb_status last = FMPB_OK;
  for (int ref = 0;; ++ref) {
    FMPB_CUDA(cudaMemcpyAsync(done, hdone.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
    if (ref > 0) FMPB_TRY(A(R, x, r, st));
    FMPB_LAUNCH("outer_residual", st, k_outer_residual<<<dim3(vb, R), 256, 0, st>>>(b, r, done, R, N, ref > 0 ? 1 : 0));
    FMPB_CUDA(cudaGetLastError());
    FMPB_TRY(norms(r, rn));
    bool all = true;
    for (int q = 0; q < R; ++q) {
      if (!hdone[q]) rel[q] = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
      if (rel[q] <= tol) hdone[q] = 1;
      all &= hdone[q] != 0;
    }
    if (all || total_it >= maxit) break;
    if (o.timeout_ms > 0 &&
        std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
            o.timeout_ms) {
      set_error("gmres_refined: wall-clock limit of %d ms reached", o.timeout_ms);
      last = FMPB_ETIMEOUT;
      break;
    }
    if (hdone != std::vector<int>(R, 0)) {
      FMPB_CUDA(cudaMemcpyAsync(done, hdone.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
      FMPB_LAUNCH("outer_residual", st, k_outer_residual<<<dim3(vb, R), 256, 0, st>>>(r, r, done, R, N, 0));
    }
    fmpb_solve_opts inner = o;
    inner.tol = inner_tol;
    inner.maxit = maxit - total_it;
    std::vector<fmpb_solve_info> ii(R);
    fmpb_status s = gmres_solve(Alow, R, N, r, d, inner, ii.data(), st, nullptr, nullptr, Alow32);
    if (s != FMPB_OK && s != FMPB_ENOCONV && s != FMPB_ETIMEOUT) return s;
    int it_max = 0;
    for (int q = 0; q < R; ++q) {
      iters[q] += ii[q].iters;
      it_max = std::max(it_max, ii[q].iters);
    }
    total_it += std::max(1, it_max);
    FMPB_LAUNCH("axpy", st, k_axpy<<<vb, 256, 0, st>>>(x, d, total));
    FMPB_CUDA(cudaGetLastError());
    ++refinements;
  }
  bool all_conv = true;
  for (int q = 0; q < R; ++q) {
    const bool conv = rel[q] <= tol;
    all_conv &= conv;
    if (info) {
      info[q].iters = iters[q];
      info[q].converged = conv ? 1 : 0;
      info[q].relres_est = rel[q];
      info[q].relres_true = rel[q];
      info[q].refinements = refinements;
    }
  }
  if (last != FMPB_OK) return last;
  if (!all_conv) {
    set_error("gmres_refined: tolerance %.3g not reached within %d inner iterations", tol, maxit);
    return FMPB_ENOCONV;
  }
  return FMPB_OK;
}

}  // namespace fmpb

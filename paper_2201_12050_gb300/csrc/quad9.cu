// Collocation blocks of the Burton-Miller operator (Sec. 2.1, Eq. (bm) and
// Eq. (matrixBEM)) on nine-node quadratic quadrilaterals with one constant
// pressure per element, collocated at the element centre: the offset blocks
// T_delta of the block Toeplitz form (Sec. 2.2, Eq. (blockToeplizMatrix)).
// The geometry, class rules and self terms are the host-and-device
// functions of quad9.cuh; here they are laid out for the device:
//   * the class-rule points of every element are expanded once into tables
//     (HBM is plentiful: 21 KB per element), the far rule point-major so
//     that a warp reading point p of 32 consecutive source elements loads
//     contiguous memory;
//   * one thread per entry (o, i, j) evaluates the far class (16 points)
//     and lists the near and very-near entries, which get a warp each (64
//     or 256 points shared by the lanes, fixed-order reduction);
//   * one warp per element evaluates the self term (the 64 angular nodes of
//     the polar rule split between the lanes).
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"

namespace fmpb {

// Element data: Q9Elem, and the collocation data (centre, normal, chord,
// area; corners 0, 2, 8 as v) in Elem for the kernels shared with triangles.
__global__ void k_q9_prepare(const double* __restrict__ nodes, const int32_t* __restrict__ elems, int n, Q9Rules R,
                             Q9Elem* __restrict__ q9, Elem* __restrict__ el) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double Y[9][3];
  for (int a = 0; a < 9; ++a) {
    const int v = elems[9 * e + a];
    for (int d = 0; d < 3; ++d) Y[a][d] = nodes[3 * v + d];
  }
  Q9Elem Q;
  q9_prepare(Y, R, Q);   // the host has checked every element
  q9[e] = Q;
  Elem E;
  const int corner[3] = {0, 2, 8};
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) E.v[a][d] = Y[corner[a]][d];
  for (int d = 0; d < 3; ++d) {
    E.c[d] = Q.c[d];
    E.nrm[d] = Q.nrm[d];
  }
  E.area = Q.area;
  E.hmax = Q.hmax;
  el[e] = E;
}

// Class-rule points of every element, thread (e, p): p < 16 the far rule,
// then the 64 near and 256 very-near points.
__global__ void k_q9_points(const Q9Elem* __restrict__ q9, int n, Q9Rules R, double* __restrict__ far_tab,
                            double* __restrict__ near_tab) {
  const int per = Q9_FAR + Q9_NEAR_TAB;
  const size_t total = (size_t)n * per;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / per), p = (int)(idx - (size_t)e * per);
    double a[9][3];
    q9_monomials(q9[e].Y, a);
    double t[7];
    if (p < Q9_FAR) {
      q9_table_point(a, R, 0, p, t);
      for (int f = 0; f < 7; ++f) far_tab[((size_t)p * 7 + f) * n + e] = t[f];
    } else {
      const int q = p - Q9_FAR;
      const int cls = q < Q9_NEAR ? 1 : 2;
      q9_table_point(a, R, cls, cls == 1 ? q : q - Q9_NEAR, t);
      double* dst = near_tab + ((size_t)e * Q9_NEAR_TAB + q) * 8;
      for (int f = 0; f < 7; ++f) dst[f] = t[f];
      dst[7] = 0.0;
    }
  }
}

// Far rule in float-float about each element's centre (the constant-pressure
// far class below): u = y - c, n_y, w|J| as (hi, lo) pairs, point-major and
// field-major like the FP64 table; thread 0 also fills the series constants.
__global__ void k_q9_far_ff(const double* __restrict__ far_tab, const Elem* __restrict__ el, int n,
                            float2* __restrict__ farff, FfConst* __restrict__ fc) {
  const size_t sn = (size_t)n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)Q9_FAR * sn;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(idx / sn), e = (int)(idx - (size_t)p * sn);
    const double* q = far_tab + (size_t)p * 7 * sn + e;
    for (int f = 0; f < 7; ++f) {
      const double v = f < 3 ? q[f * sn] - el[e].c[f] : q[f * sn];
      const ff w = ff_from_d(v);
      farff[((size_t)p * 7 + f) * sn + e] = make_float2(w.h, w.l);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    FfConst C{};
    ff_const_series(C);
    *fc = C;
  }
}

// D, H (S, K) of a far constant-pressure element j in float-float (the
// triangles' far class, here with the curved element's per-point normal):
// FP64 keeps e = x - (c + shift), |e| and the reference phase k|e| mod 2 pi;
// per point u = y - c, Delta = |u|^2 - 2 e.u, r = sqrt(|e|^2 + Delta),
// delta = Delta / (|e| + r), e^{ikr} = e^{ik|e|} e^{ik delta}.
template <bool SK>
__device__ void q9_far_ff(const float2* __restrict__ tab, size_t sn, int j, const double dc[3], double dist,
                          const double nx[3], double k, double hmax, const FfConst& C, cd& D, cd& H, cd& S,
                          cd& K) {
  const ff ef[3] = {ff_from_d(dc[0]), ff_from_d(dc[1]), ff_from_d(dc[2])};
  const ff nxf[3] = {ff_from_d(nx[0]), ff_from_d(nx[1]), ff_from_d(nx[2])};
  const ff kf = ff_from_d(k);
  const ff rho2 = ff_dot3(ef, ef);
  const ff rho = ff_sqrt(rho2);
  const ff enx = ff_dot3(ef, nxf);
  double th = k * dist;
  const double qn = rint(th * (1.0 / TWO_PI_HI));
  th = fma(-qn, TWO_PI_HI, th);
  th = fma(-qn, TWO_PI_LO, th);
  const ffc Eref = expi_ff(ff_from_d(th), 3, C);
  // |k delta| <= k |u| <= 1.5 k hmax on the curved element
  int m = 2;
  const float kh = (float)(1.5 * k * hmax);
  while (kh > 0.75f * (float)(1 << m) && m < 12) ++m;
  ff Dre = ff_make(0.f), Dim = ff_make(0.f), Hre = ff_make(0.f), Him = ff_make(0.f);
  ff Sre = ff_make(0.f), Sim = ff_make(0.f), Kre = ff_make(0.f), Kim = ff_make(0.f);
#pragma unroll 1
  for (int p = 0; p < Q9_FAR; ++p) {
    const float2* q = tab + (size_t)p * 7 * sn + j;
    ff u[3], ny[3];
    for (int d = 0; d < 3; ++d) {
      const float2 a = q[d * sn], b = q[(3 + d) * sn];
      u[d] = ff{a.x, a.y};
      ny[d] = ff{b.x, b.y};
    }
    const float2 wq = q[6 * sn];
    const ff w = ff{wq.x, wq.y};
    const ff eu = ff_dot3(ef, u);
    const ff Delta = ff_sub(ff_dot3(u, u), ff{2.f * eu.h, 2.f * eu.l});
    const ff r = ff_sqrt(ff_add(rho2, Delta));
    const ff delta = ff_div(Delta, ff_add(rho, r));
    const ffc E = ffc_mul(Eref, expi_ff(ff_mul(kf, delta), m, C));
    const ff ir = ff_rcp(r);
    const ff ir2 = ff_mul(ir, ir);
    const ff ir3 = ff_mul(ir2, ir);
    const ff ir5 = ff_mul(ir3, ir2);
    const ff kr = ff_mul(kf, r);
    // x - y = e - u
    const ff dny = ff_sub(ff_dot3(ef, ny), ff_dot3(u, ny));
    const ff dnx = ff_sub(enx, ff_dot3(u, nxf));
    const ff nn = ff_dot3(nxf, ny);
    const ff are = ff_add(E.re, ff_mul(E.im, kr));
    const ff aim = ff_sub(E.im, ff_mul(E.re, kr));
    const ff t3 = ff_sub(ff_make(3.f), ff_mul(kr, kr));
    const ff kr3 = ff_mul_f(kr, 3.f);
    const ff bre = ff_add(ff_mul(E.re, t3), ff_mul(E.im, kr3));
    const ff bim = ff_sub(ff_mul(E.im, t3), ff_mul(E.re, kr3));
    const ff wi = ff_mul(w, C.inv4pi);
    const ff wir3 = ff_mul(wi, ir3);
    const ff f = ff_mul(wir3, dny);
    const ff g1 = ff_mul(wir3, nn);
    const ff g2 = ff_mul(ff_mul(ff_mul(wi, ir5), dnx), dny);
    Dre = ff_add(Dre, ff_mul(are, f));
    Dim = ff_add(Dim, ff_mul(aim, f));
    Hre = ff_add(Hre, ff_sub(ff_mul(are, g1), ff_mul(bre, g2)));
    Him = ff_add(Him, ff_sub(ff_mul(aim, g1), ff_mul(bim, g2)));
    if (SK) {
      const ff gs = ff_mul(wi, ir);
      Sre = ff_add(Sre, ff_mul(E.re, gs));
      Sim = ff_add(Sim, ff_mul(E.im, gs));
      const ff gk = ff_mul(wir3, dnx);
      Kre = ff_sub(Kre, ff_mul(are, gk));
      Kim = ff_sub(Kim, ff_mul(aim, gk));
    }
  }
  D = mkc(ff_to_d(Dre), ff_to_d(Dim));
  H = mkc(ff_to_d(Hre), ff_to_d(Him));
  if (SK) {
    S = mkc(ff_to_d(Sre), ff_to_d(Sim));
    K = mkc(ff_to_d(Kre), ff_to_d(Kim));
  }
}

// One thread per entry (o, i, j) of n_off blocks of n x n; block o goes to
// out + dest[o] n n.  The diagonal of the zero offset is left to k_q9_self.
// Far entries are summed here; near and very-near entries are listed for
// k_q9_near_entries, or summed here when the list is full.
template <bool SK>
__global__ void __launch_bounds__(128) k_q9_blocks(const Elem* __restrict__ el, const double* __restrict__ far_tab,
                                                   const float2* __restrict__ far_ff,
                                                   const FfConst* __restrict__ fc,
                                                   const double* __restrict__ near_tab, int n,
                                                   const double* __restrict__ shifts,
                                                   const int64_t* __restrict__ dest, int n_off, int zero_off,
                                                   cd* __restrict__ out, double k, cd beta, BlockWrite bw,
                                                   unsigned long long* __restrict__ near_list,
                                                   unsigned long long* __restrict__ near_count,
                                                   unsigned long long near_cap) {
  const size_t nn = (size_t)n * n;
  const size_t total = nn * (size_t)n_off;
  const size_t sn = (size_t)n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx / nn);
    const size_t rem = idx - (size_t)o * nn;
    const int i = (int)(rem / n);
    const int j = (int)(rem - (size_t)i * n);
    if (o == zero_off && i == j) continue;
    const Elem& Ti = el[i];
    const double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    const double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const Elem& Ej = el[j];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (Ej.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    cd D = mkc(0.0, 0.0), H = mkc(0.0, 0.0), S = mkc(0.0, 0.0), K = mkc(0.0, 0.0);
    if (dist >= FAR_RATIO * Ej.hmax) {
      if (far_ff) {
        q9_far_ff<SK>(far_ff, sn, j, dc, dist, nx, k, Ej.hmax, *fc, D, H, S, K);
      } else {
#pragma unroll 1
        for (int p = 0; p < Q9_FAR; ++p) {
          const double* q = far_tab + (size_t)p * 7 * sn + j;
          const double dv[3] = {x[0] - (q[0] + sh[0]), x[1] - (q[sn] + sh[1]), x[2] - (q[2 * sn] + sh[2])};
          const double ny[3] = {q[3 * sn], q[4 * sn], q[5 * sn]};
          q9_kernels<SK>(dv, nx, ny, q[6 * sn], k, D, H, S, K);
        }
      }
    } else {
      if (near_list) {
        const unsigned long long slot = atomicAdd(near_count, 1ull);
        if (slot < near_cap) {
          near_list[slot] = idx;
          continue;
        }
      }
      const bool very = dist < NEAR_RATIO * Ej.hmax;
      const double* tab = near_tab + (size_t)j * Q9_NEAR_TAB * 8 + (very ? Q9_NEAR * 8 : 0);
      q9_sum_table<SK>(tab, very ? Q9_VNEAR : Q9_NEAR, 0, 1, x, nx, sh, k, D, H, S, K);
    }
    bw.put(out + (size_t)dest[o] * nn + rem, SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k));
  }
}

// Near and very-near entries listed by k_q9_blocks, one warp per entry.
template <bool SK>
__global__ void __launch_bounds__(256) k_q9_near_entries(const Elem* __restrict__ el,
                                                         const double* __restrict__ near_tab, int n,
                                                         const double* __restrict__ shifts,
                                                         const int64_t* __restrict__ dest,
                                                         const unsigned long long* __restrict__ list,
                                                         const unsigned long long* __restrict__ count,
                                                         unsigned long long cap, cd* __restrict__ out, double k,
                                                         cd beta, BlockWrite bw) {
  const size_t nn = (size_t)n * n;
  const unsigned long long total = min(*count, cap);
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long w = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
       w += nwarps) {
    const size_t idx = list[w];
    const int o = (int)(idx / nn);
    const size_t rem = idx - (size_t)o * nn;
    const int i = (int)(rem / n);
    const int j = (int)(rem - (size_t)i * n);
    const Elem& Ti = el[i];
    const Elem& Ej = el[j];
    const double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    const double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (Ej.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    const bool very = dist < NEAR_RATIO * Ej.hmax;
    const double* tab = near_tab + (size_t)j * Q9_NEAR_TAB * 8 + (very ? Q9_NEAR * 8 : 0);
    cd D = mkc(0.0, 0.0), H = mkc(0.0, 0.0), S = mkc(0.0, 0.0), K = mkc(0.0, 0.0);
    q9_sum_table<SK>(tab, very ? Q9_VNEAR : Q9_NEAR, lane, 32, x, nx, sh, k, D, H, S, K);
    for (int off = 16; off > 0; off >>= 1) {
      D.x += __shfl_xor_sync(0xffffffffu, D.x, off);
      D.y += __shfl_xor_sync(0xffffffffu, D.y, off);
      H.x += __shfl_xor_sync(0xffffffffu, H.x, off);
      H.y += __shfl_xor_sync(0xffffffffu, H.y, off);
      if (SK) {
        S.x += __shfl_xor_sync(0xffffffffu, S.x, off);
        S.y += __shfl_xor_sync(0xffffffffu, S.y, off);
        K.x += __shfl_xor_sync(0xffffffffu, K.x, off);
        K.y += __shfl_xor_sync(0xffffffffu, K.y, off);
      }
    }
    if (lane == 0)
      bw.put(out + (size_t)dest[o] * nn + rem, SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k));
  }
}

// Self term of every element, one warp per element:
// T_ii = 1/2 + beta/2 - (D + (i/k) H) - i k beta (S + (i/k) K) at the centre,
// stored at block0[i n + i], or with slot at block0[slot[i]] (listed
// entries; -1: not listed).
template <bool SK>
__global__ void __launch_bounds__(256) k_q9_self(const Q9Elem* __restrict__ q9, int n, cd* __restrict__ block0,
                                                 double k, cd beta, Q9Rules R, const int64_t* __restrict__ slot) {
  const int lane = threadIdx.x & 31;
  const int e = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (e >= n) return;   // uniform across the warp
  Q9Centre C;
  q9_centre(q9[e].Y, C);
  cd D = mkc(0.0, 0.0), H = mkc(0.0, 0.0), S = mkc(0.0, 0.0), K = mkc(0.0, 0.0);
  for (int it = lane; it < Q9_THETA; it += 32) q9_self_theta<SK>(C, R, k, it, D, H, S, K);
  for (int off = 16; off > 0; off >>= 1) {
    D.x += __shfl_xor_sync(0xffffffffu, D.x, off);
    D.y += __shfl_xor_sync(0xffffffffu, D.y, off);
    H.x += __shfl_xor_sync(0xffffffffu, H.x, off);
    H.y += __shfl_xor_sync(0xffffffffu, H.y, off);
    if (SK) {
      S.x += __shfl_xor_sync(0xffffffffu, S.x, off);
      S.y += __shfl_xor_sync(0xffffffffu, S.y, off);
      K.x += __shfl_xor_sync(0xffffffffu, K.x, off);
      K.y += __shfl_xor_sync(0xffffffffu, K.y, off);
    }
  }
  if (lane == 0) {
    const cd t = cadd(SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k), mkc(0.5 + 0.5 * beta.x, 0.5 * beta.y));
    if (!slot)
      block0[(size_t)e * n + e] = t;
    else if (slot[e] >= 0)
      block0[slot[e]] = t;
  }
}

// Listed entries (o, i, j) of n_off blocks (idx = (o n + i) n + j), written
// to out[e]: the exact entries a multilevel near field keeps.  Same classes
// and arithmetic as k_q9_blocks, near classes in the thread itself; the self
// entry of the zero offset is left to k_q9_self.
template <bool SK>
__global__ void __launch_bounds__(128) k_q9_entries(const Elem* __restrict__ el, const double* __restrict__ far_tab,
                                                    const double* __restrict__ near_tab, int n,
                                                    const double* __restrict__ shifts, int zero_off,
                                                    const int64_t* __restrict__ list, int64_t count,
                                                    cd* __restrict__ out, double k, cd beta) {
  const size_t nn = (size_t)n * n;
  const size_t sn = (size_t)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const size_t idx = (size_t)list[e];
    const int o = (int)(idx / nn);
    const size_t rem = idx - (size_t)o * nn;
    const int i = (int)(rem / n);
    const int j = (int)(rem - (size_t)i * n);
    if (o == zero_off && i == j) continue;
    const Elem& Ti = el[i];
    const double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    const double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const Elem& Ej = el[j];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (Ej.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    cd D = mkc(0.0, 0.0), H = mkc(0.0, 0.0), S = mkc(0.0, 0.0), K = mkc(0.0, 0.0);
    if (dist >= FAR_RATIO * Ej.hmax) {
#pragma unroll 1
      for (int p = 0; p < Q9_FAR; ++p) {
        const double* q = far_tab + (size_t)p * 7 * sn + j;
        const double dv[3] = {x[0] - (q[0] + sh[0]), x[1] - (q[sn] + sh[1]), x[2] - (q[2 * sn] + sh[2])};
        const double ny[3] = {q[3 * sn], q[4 * sn], q[5 * sn]};
        q9_kernels<SK>(dv, nx, ny, q[6 * sn], k, D, H, S, K);
      }
    } else {
      const bool very = dist < NEAR_RATIO * Ej.hmax;
      const double* tab = near_tab + (size_t)j * Q9_NEAR_TAB * 8 + (very ? Q9_NEAR * 8 : 0);
      q9_sum_table<SK>(tab, very ? Q9_VNEAR : Q9_NEAR, 0, 1, x, nx, sh, k, D, H, S, K);
    }
    out[e] = SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k);
  }
}

// ------------------------------------------------------------ host side --
static Q9Rules q9_rules() {
  Q9Rules R;
  for (int i = 0; i < 4; ++i) gl_node(4, i, &R.t4[i], &R.w4[i]);
  for (int i = 0; i < 8; ++i) gl_node(8, i, &R.t8[i], &R.w8[i]);
  for (int i = 0; i < 16; ++i) gl_node(16, i, &R.t16[i], &R.w16[i]);
  for (int i = 0; i < 24; ++i) gl_node(24, i, &R.t24[i], &R.w24[i]);
  return R;
}

fmpb_status upload_mesh_q9(const double* nodes, int64_t nn, const int32_t* elems, int64_t n, DeviceMesh& m,
                           cudaStream_t st) {
  if (!nodes || !elems || nn < 9 || n < 1 || n > (1 << 20)) {
    set_error("mesh: need nodes (nn >= 9) and quadrilaterals (1 <= n <= 2^20)");
    return FMPB_EINVAL;
  }
  for (int64_t e = 0; e < 3 * nn; ++e)
    if (!std::isfinite(nodes[e])) {
      set_error("mesh: node coordinate %lld is not finite", (long long)e);
      return FMPB_EMESH;
    }
  const Q9Rules R = q9_rules();
  double rho = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    double Y[9][3];
    for (int a = 0; a < 9; ++a) {
      const int32_t v = elems[9 * t + a];
      if (v < 0 || v >= nn) {
        set_error("mesh: quadrilateral %lld references node %d (nn = %lld)", (long long)t, v, (long long)nn);
        return FMPB_EMESH;
      }
      for (int d = 0; d < 3; ++d) Y[a][d] = nodes[3 * (int64_t)v + d];
      rho = fmax(rho, sqrt(Y[a][0] * Y[a][0] + Y[a][1] * Y[a][1] + Y[a][2] * Y[a][2]));
    }
    Q9Elem E;
    if (!q9_prepare(Y, R, E)) {
      set_error("mesh: quadrilateral %lld is degenerate (vanishing Jacobian)", (long long)t);
      return FMPB_EMESH;
    }
  }
  m.n = (int)n;
  m.nodes = 9;
  m.q9r = R;
  m.radius = rho;
  double* dnodes = nullptr;
  int32_t* delems = nullptr;
  FMPB_CUDA(cudaMalloc(&dnodes, sizeof(double) * 3 * nn));
  cudaError_t e = cudaMalloc(&delems, sizeof(int32_t) * 9 * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.el, sizeof(Elem) * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.q9, sizeof(Q9Elem) * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.q9_far, sizeof(double) * Q9_FAR * 7 * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.q9_near, sizeof(double) * Q9_NEAR_TAB * 8 * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.q9_farff, sizeof(float2) * Q9_FAR * 7 * n);
  if (e == cudaSuccess) e = cudaMalloc(&m.fc_dev, sizeof(FfConst));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dnodes, nodes, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(delems, elems, sizeof(int32_t) * 9 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    FMPB_LAUNCH("q9_prepare", st, k_q9_prepare<<<grid_for(n, 128), 128, 0, st>>>(dnodes, delems, (int)n, R, m.q9, m.el));
    const size_t pts = (size_t)n * (Q9_FAR + Q9_NEAR_TAB);
    FMPB_LAUNCH("q9_points", st, k_q9_points<<<(unsigned)std::min<size_t>(grid_for(pts, 256), 152 * 32), 256, 0, st>>>(m.q9, (int)n, R, m.q9_far, m.q9_near));
    FMPB_LAUNCH("q9_far_ff", st, k_q9_far_ff<<<(unsigned)std::min<size_t>(grid_for((size_t)n * Q9_FAR, 256), 152 * 32), 256, 0, st>>>(m.q9_far, m.el, (int)n, m.q9_farff, m.fc_dev));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dnodes);
  cudaFree(delems);
  if (e != cudaSuccess) return cuda_status(e, "upload_mesh_q9");
  return FMPB_OK;
}

fmpb_status build_blocks_q9(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                            const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st) {
  if (m.nodes != 9 || !m.q9) {
    set_error("build_blocks_q9: not a nine-node mesh");
    return FMPB_EINVAL;
  }
  if (m.q9_order > 0) return build_blocks_q9p(m, g, k, beta, n_off, offsets, dest_host, out, st);
  std::vector<double> shifts(3 * (size_t)n_off);
  int zero_off = -1;
  for (int o = 0; o < n_off; ++o) {
    const int32_t* dl = offsets + 3 * o;
    if (dl[0] == 0 && dl[1] == 0 && dl[2] == 0) zero_off = o;
    for (int d = 0; d < 3; ++d) shifts[3 * o + d] = -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
  }
  const BlockWrite bw{mkc(1.0, 0.0), 0, 0};
  double* dshift = nullptr;
  int64_t* ddest = nullptr;
  FMPB_CUDA(cudaMalloc(&dshift, sizeof(double) * 3 * n_off));
  cudaError_t e = cudaMalloc(&ddest, sizeof(int64_t) * n_off);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dshift, shifts.data(), sizeof(double) * 3 * n_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ddest, dest_host, sizeof(int64_t) * n_off, cudaMemcpyHostToDevice, st);
  const size_t total = (size_t)m.n * m.n * n_off;
  const unsigned long long near_cap = (unsigned long long)std::min<size_t>(total, (size_t)8 << 20);
  unsigned long long* near_list = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&near_list, sizeof(unsigned long long) * (near_cap + 1));
  unsigned long long* near_count = near_list ? near_list + near_cap : nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(near_count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)std::min<size_t>(grid_for(total, 128), (size_t)152 * 64);
    const unsigned self_blocks = grid_for((size_t)m.n * 32, 256);
    if (beta.x == 0.0 && beta.y == 0.0) {
      FMPB_LAUNCH("q9_blocks", st, k_q9_blocks<false><<<blocks, 128, 0, st>>>(m.el, m.q9_far, m.q9_farff, m.fc_dev, m.q9_near, m.n, dshift, ddest, n_off, zero_off, out, k, beta, bw, near_list, near_count, near_cap));
      FMPB_LAUNCH("q9_near", st, k_q9_near_entries<false><<<152 * 16, 256, 0, st>>>(m.el, m.q9_near, m.n, dshift, ddest, near_list, near_count, near_cap, out, k, beta, bw));
      if (zero_off >= 0)
        FMPB_LAUNCH("q9_self", st, k_q9_self<false><<<self_blocks, 256, 0, st>>>(m.q9, m.n, out + (size_t)dest_host[zero_off] * m.n * m.n, k, beta, m.q9r, nullptr));
    } else {
      FMPB_LAUNCH("q9_blocks_adm", st, k_q9_blocks<true><<<blocks, 128, 0, st>>>(m.el, m.q9_far, m.q9_farff, m.fc_dev, m.q9_near, m.n, dshift, ddest, n_off, zero_off, out, k, beta, bw, near_list, near_count, near_cap));
      FMPB_LAUNCH("q9_near_adm", st, k_q9_near_entries<true><<<152 * 16, 256, 0, st>>>(m.el, m.q9_near, m.n, dshift, ddest, near_list, near_count, near_cap, out, k, beta, bw));
      if (zero_off >= 0)
        FMPB_LAUNCH("q9_self_adm", st, k_q9_self<true><<<self_blocks, 256, 0, st>>>(m.q9, m.n, out + (size_t)dest_host[zero_off] * m.n * m.n, k, beta, m.q9r, nullptr));
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dshift);
  cudaFree(ddest);
  cudaFree(near_list);
  if (e != cudaSuccess) return cuda_status(e, "build_blocks_q9");
  return FMPB_OK;
}

}  // namespace fmpb

namespace fmpb {

fmpb_status build_entries_q9(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                             const int32_t* offsets, const int64_t* list, int64_t count, const int64_t* self_slot,
                             cd* out, cudaStream_t st) {
  if (m.nodes != 9 || !m.q9 || m.q9_order != 0) {
    set_error("build_entries: listed entries take flat triangles or constant pressure on nine-node elements");
    return FMPB_EINVAL;
  }
  std::vector<double> shifts(3 * (size_t)n_off);
  int zero_off = -1;
  for (int o = 0; o < n_off; ++o) {
    const int32_t* dl = offsets + 3 * o;
    if (dl[0] == 0 && dl[1] == 0 && dl[2] == 0) zero_off = o;
    for (int d = 0; d < 3; ++d) shifts[3 * o + d] = -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
  }
  double* dshift = nullptr;
  FMPB_CUDA(cudaMallocAsync(&dshift, sizeof(double) * 3 * n_off, st));
  FMPB_CUDA(cudaMemcpyAsync(dshift, shifts.data(), sizeof(double) * 3 * n_off, cudaMemcpyHostToDevice, st));
  if (count > 0) {
    const unsigned blocks = (unsigned)std::min<int64_t>((count + 127) / 128, 152 * 64);
    if (beta.x == 0.0 && beta.y == 0.0)
      FMPB_LAUNCH("q9_entries", st, k_q9_entries<false><<<blocks, 128, 0, st>>>(m.el, m.q9_far, m.q9_near, m.n, dshift, zero_off, list, count, out, k, beta));
    else
      FMPB_LAUNCH("q9_entries_adm", st, k_q9_entries<true><<<blocks, 128, 0, st>>>(m.el, m.q9_far, m.q9_near, m.n, dshift, zero_off, list, count, out, k, beta));
  }
  if (zero_off >= 0 && self_slot) {
    const unsigned self_blocks = grid_for((size_t)m.n * 32, 256);
    if (beta.x == 0.0 && beta.y == 0.0)
      FMPB_LAUNCH("q9_self", st, k_q9_self<false><<<self_blocks, 256, 0, st>>>(m.q9, m.n, out, k, beta, m.q9r, self_slot));
    else
      FMPB_LAUNCH("q9_self_adm", st, k_q9_self<true><<<self_blocks, 256, 0, st>>>(m.q9, m.n, out, k, beta, m.q9r, self_slot));
  }
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaFreeAsync(dshift, st));
  return FMPB_OK;
}

}  // namespace fmpb

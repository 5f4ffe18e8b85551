// Collocation quadrature of the Burton-Miller operator for a rigid boundary
// (Sec. 2.1, Eq. (bm) with dp/dn = 0) on flat triangles with constant
// pressure: the offset blocks T_delta of the multilevel block Toeplitz form
// (Sec. 2.2, Eq. (blockToeplizMatrix)), which are also the near-field blocks
// S_delta of the FMPBEM (Sec. 3.2), the singular self term, the plane-wave
// right-hand side and the field-point evaluation (Eq. (cbie), c = 1).
//
// Mesh normals n_m point into the fluid, the opposite of the paper's n, so
//   T_delta[i][j] = 1/2 [self] - (D_ij + (i/k) H_ij),
//   D_ij = int_{E_j} dG/dn_y,  H_ij = int_{E_j} d2G/dn_x dn_y  (mesh normals),
// G = e^{ikr}/(4 pi r) (Eq. (green3dFull)).
//
// Quadrature rule (the operator's definition; d = |x_i - centroid_j|,
// h = longest edge of E_j; thresholds scaled by 1 + 1e-9, ties to the more
// accurate class):
//   d >= 4h        collapsed Gauss-Legendre 3x3 with apex v0,
//   1.5h <= d < 4h collapsed 8x8,
//   d < 1.5h       collapsed 8x8 on each of the four midpoint children,
//   self           closed-form Hadamard finite part of r^-3 plus the polar
//                  8x8 remainder on the children (x, v_a, v_b).
// Collapsed rule of order q on (a, b, c): y(s,t) = a + s[(b-a) + t(c-b)],
// dA = 2 area s ds dt, Gauss-Legendre nodes in s and t.
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "ff.cuh"

namespace fmpb {

// ------------------------------------------------------------ geometry ----
__global__ void k_prepare_elements(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                                   int n, Elem* __restrict__ el) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  Elem E;
  for (int a = 0; a < 3; ++a) {
    int vid = tris[3 * e + a];
    for (int d = 0; d < 3; ++d) E.v[a][d] = verts[3 * vid + d];
  }
  double e1[3], e2[3], cr[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = E.v[1][d] - E.v[0][d];
    e2[d] = E.v[2][d] - E.v[0][d];
  }
  cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
  cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
  cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  E.area = 0.5 * len;
  for (int d = 0; d < 3; ++d) {
    E.nrm[d] = cr[d] / len;
    E.c[d] = (E.v[0][d] + E.v[1][d] + E.v[2][d]) / 3.0;
  }
  double h = 0.0;
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3;
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      double t = E.v[b][d] - E.v[a][d];
      s += t * t;
    }
    h = fmax(h, sqrt(s));
  }
  E.hmax = h;
  el[e] = E;
}

// Gauss-Legendre nodes/weights on [0,1] by Newton's method on P_q (three-term
// recurrence), one thread per node.
__host__ __device__ void gl_node(int q, int i, double* t, double* w) {
  double x = cos(PI * (i + 0.75) / (q + 0.5));
  double p0 = 1.0, p1 = x, dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    p0 = 1.0;
    p1 = x;
    for (int n = 2; n <= q; ++n) {
      double p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    dp = q * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  p0 = 1.0;
  p1 = x;
  for (int n = 2; n <= q; ++n) {
    double p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
    p0 = p1;
    p1 = p2;
  }
  dp = q * (x * p1 - p0) / (x * x - 1.0);
  *t = 0.5 * (1.0 - x);                    // ascending order on [0, 1]
  *w = 1.0 / ((1.0 - x * x) * dp * dp);    // 2/((1-x^2) P_q'^2), halved for [0, 1]
}

__global__ void k_gauss_legendre(QuadRules* qr) {
  int i = threadIdx.x;
  if (i < Q_FAR) gl_node(Q_FAR, i, &qr->t3[i], &qr->w3[i]);
  if (i < Q_NEAR) gl_node(Q_NEAR, i, &qr->t8[i], &qr->w8[i]);
}

// ------------------------------------------------------------- kernels ----
// Accumulates w*dG/dn_y into D and w*d2G/dn_x dn_y into H at one point, and
// with SK also w*G into S and w*dG/dn_x into K (admittance boundaries).
template <bool SK>
__device__ __forceinline__ void kernel_point4(const double x[3], const double nx[3], const double y[3],
                                              const double ny[3], double w, double k, cd& D, cd& H, cd& S,
                                              cd& K) {
  const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
  const double r = sqrt(r2);
  const double ir = 1.0 / r;
  const double kr = k * r;
  double s, c;
  sincos(kr, &s, &c);
  const double dny = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
  const double dnx = d0 * nx[0] + d1 * nx[1] + d2 * nx[2];
  const double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
  const double inv4pi = 0.25 / PI;
  const double ir3 = ir * ir * ir;
  // e^{ikr}(1 - ikr)
  const double a_re = c + s * kr, a_im = s - c * kr;
  const double f = w * dny * ir3 * inv4pi;
  D.x = fma(a_re, f, D.x);
  D.y = fma(a_im, f, D.y);
  // e^{ikr}(3 - k^2 r^2 - 3ikr)
  const double t = 3.0 - kr * kr;
  const double b_re = c * t + 3.0 * s * kr, b_im = s * t - 3.0 * c * kr;
  const double g1 = w * nn * ir3 * inv4pi;
  const double g2 = w * dnx * dny * ir3 * ir * ir * inv4pi;
  H.x += a_re * g1 - b_re * g2;
  H.y += a_im * g1 - b_im * g2;
  if (SK) {
    // G = e^{ikr} / (4 pi r),  dG/dn_x = -e^{ikr}(1 - ikr) ((x-y).n_x) / (4 pi r^3)
    const double gs = w * ir * inv4pi;
    S.x = fma(c, gs, S.x);
    S.y = fma(s, gs, S.y);
    const double gk = -w * dnx * ir3 * inv4pi;
    K.x = fma(a_re, gk, K.x);
    K.y = fma(a_im, gk, K.y);
  }
}
__device__ __forceinline__ void kernel_point(const double x[3], const double nx[3], const double y[3],
                                             const double ny[3], double w, double k, cd& D, cd& H) {
  cd S, K;
  kernel_point4<false>(x, nx, y, ny, w, k, D, H, S, K);
}

template <int Q, bool SK>
__device__ __forceinline__ void integrate_collapsed(const double a[3], const double b[3], const double cc[3],
                                                    double two_area, const double* t, const double* w,
                                                    const double x[3], const double nx[3], const double ny[3],
                                                    double k, cd& D, cd& H, cd& S, cd& K) {
  double ba[3], cb[3];
  for (int d = 0; d < 3; ++d) {
    ba[d] = b[d] - a[d];
    cb[d] = cc[d] - b[d];
  }
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    const double s = t[i];
    const double ws = two_area * s * w[i];
#pragma unroll 1
    for (int j = 0; j < Q; ++j) {
      double y[3];
      for (int d = 0; d < 3; ++d) y[d] = a[d] + s * (ba[d] + t[j] * cb[d]);
      kernel_point4<SK>(x, nx, y, ny, ws * w[j], k, D, H, S, K);
    }
  }
}

// D, H of element E (translated by shift) seen from (x, nx), by class.  Kept
// out of line with rolled loops: the quadrature kernel's code must stay small
// enough for the instruction cache, and these classes are a few per cent of
// the points.
template <bool SK>
__device__ void element_dh_t(const Elem& E, const double shift[3], const double x[3], const double nx[3],
                             double k, const QuadRules& qr, cd& D, cd& H, cd& S, cd& K) {
  double v[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) v[a][d] = E.v[a][d] + shift[d];
  double dc[3];
  for (int d = 0; d < 3; ++d) dc[d] = x[d] - (E.c[d] + shift[d]);
  const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
  const double two_area = 2.0 * E.area;
  D = mkc(0.0, 0.0);
  H = mkc(0.0, 0.0);
  S = mkc(0.0, 0.0);
  K = mkc(0.0, 0.0);
  if (dist >= FAR_RATIO * E.hmax) {
    integrate_collapsed<Q_FAR, SK>(v[0], v[1], v[2], two_area, qr.t3, qr.w3, x, nx, E.nrm, k, D, H, S, K);
  } else if (dist >= NEAR_RATIO * E.hmax) {
    integrate_collapsed<Q_NEAR, SK>(v[0], v[1], v[2], two_area, qr.t8, qr.w8, x, nx, E.nrm, k, D, H, S, K);
  } else {
    double m01[3], m12[3], m20[3];
    for (int d = 0; d < 3; ++d) {
      m01[d] = 0.5 * (v[0][d] + v[1][d]);
      m12[d] = 0.5 * (v[1][d] + v[2][d]);
      m20[d] = 0.5 * (v[2][d] + v[0][d]);
    }
    const double ta = 0.25 * two_area;
    integrate_collapsed<Q_NEAR, SK>(v[0], m01, m20, ta, qr.t8, qr.w8, x, nx, E.nrm, k, D, H, S, K);
    integrate_collapsed<Q_NEAR, SK>(m01, v[1], m12, ta, qr.t8, qr.w8, x, nx, E.nrm, k, D, H, S, K);
    integrate_collapsed<Q_NEAR, SK>(m20, m12, v[2], ta, qr.t8, qr.w8, x, nx, E.nrm, k, D, H, S, K);
    integrate_collapsed<Q_NEAR, SK>(m01, m12, m20, ta, qr.t8, qr.w8, x, nx, E.nrm, k, D, H, S, K);
  }
}
__device__ __noinline__ void element_dh(const Elem& E, const double shift[3], const double x[3], const double nx[3],
                                        double k, const QuadRules& qr, cd& D, cd& H) {
  cd S, K;
  element_dh_t<false>(E, shift, x, nx, k, qr, D, H, S, K);
}
__device__ __noinline__ void element_dhsk(const Elem& E, const double shift[3], const double x[3],
                                          const double nx[3], double k, const QuadRules& qr, cd& D, cd& H, cd& S,
                                          cd& K) {
  element_dh_t<true>(E, shift, x, nx, k, qr, D, H, S, K);
}

// ------------------------------------------------- float-float far rule --
// The far class (d >= 4h, 9 points, about 97 % of all quadrature points) is
// evaluated in float-float arithmetic on the FP32 pipe.  FP64 keeps the parts
// that need it: the class decision, e = x - c (c = element centroid) and the
// reference phase k|e| reduced mod 2 pi.  Per point, with u = y - c,
//   Delta = |u|^2 - 2 e.u,   r = sqrt(|e|^2 + Delta),   delta = Delta/(|e| + r),
//   e^{ikr} = e^{ik|e|} e^{ik delta},
// so only the small phase k delta (|k delta| <= k h) is formed per point;
// e^{i psi} comes from Taylor series at psi / 2^m (|psi / 2^m| <= 0.75,
// nine terms) followed by m complex squarings.

// Per-element geometry in float-float (source side, shift free).
__global__ void k_prepare_ff(const Elem* __restrict__ el, int n, FfElem* __restrict__ fe, const QuadRules* qr,
                             FfConst* fc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const Elem E = el[e];
    FfElem F;
    for (int d = 0; d < 3; ++d) {
      F.w0[d] = ff_from_d(E.v[0][d] - E.c[d]);
      F.ba[d] = ff_from_d(E.v[1][d] - E.v[0][d]);
      F.cb[d] = ff_from_d(E.v[2][d] - E.v[1][d]);
      F.ny[d] = ff_from_d(E.nrm[d]);
      F.c[d] = ff_from_d(E.c[d]);
    }
    F.two_area = ff_from_d(2.0 * E.area);
    F.hmax = (float)E.hmax;
    F.pad = 0.f;
    fe[e] = F;
  }
  if (e == 0) {
    FfConst C;
    for (int i = 0; i < Q_FAR; ++i) {
      C.s[i] = ff_from_d(qr->t3[i]);
      C.t[i] = ff_from_d(qr->t3[i]);
      for (int j = 0; j < Q_FAR; ++j) C.W[i * Q_FAR + j] = ff_from_d(qr->t3[i] * qr->w3[i] * qr->w3[j]);
    }
    ff_const_series(C);
    *fc = C;
  }
}

// D, H (and with SK also S, K) of a far element as float-float sums
// acc = {Re D, Im D, Re H, Im H, Re S, Im S, Re K, Im K}.  ef = x - (c + shift)
// in float-float (formed on the FP32 pipe from float-float centroids and
// shift; about 1e-13 relative to |e| >= 4 h), dist = |e| in FP64 for the
// reference phase.
template <bool SK>
__device__ void far_sums_ff(const FfElem& F, const ff ef[3], double dist, const ff nxf[3], double k, ff kf,
                            const FfConst& C, ff (&acc)[8]) {
  const ff rho2 = ff_dot3(ef, ef);
  const ff rho = ff_sqrt(rho2);
  const ff dny = ff_dot3(ef, F.ny);           // (x - y).n_y is constant on the flat element
  const ff enx = ff_dot3(ef, nxf);
  const ff Cd = ff_mul(dny, C.inv4pi);
  const ff Cg1 = ff_mul(ff_dot3(nxf, F.ny), C.inv4pi);
  const ff w0nx = ff_dot3(F.w0, nxf), banx = ff_dot3(F.ba, nxf), cbnx = ff_dot3(F.cb, nxf);
  // reference phase k|e| reduced to [-pi, pi] in FP64
  double th = k * dist;
  const double qn = rint(th * (1.0 / TWO_PI_HI));
  th = fma(-qn, TWO_PI_HI, th);
  th = fma(-qn, TWO_PI_LO, th);
  const ffc Eref = expi_ff(ff_from_d(th), 3, C);
  int m = 2;
  const float kh = (float)k * F.hmax;
  while (kh > 0.75f * (float)(1 << m) && m < 12) ++m;
  ff Dre = ff_make(0.f), Dim = ff_make(0.f), Hre = ff_make(0.f), Him = ff_make(0.f);
  ff Sre = ff_make(0.f), Sim = ff_make(0.f), Kre = ff_make(0.f), Kim = ff_make(0.f);
#pragma unroll 1
  for (int b = 0; b < Q_FAR; ++b) {
    ff qb[3];
    for (int d = 0; d < 3; ++d) qb[d] = ff_add(F.ba[d], ff_mul(C.t[b], F.cb[d]));
    const ff qnx = ff_add(banx, ff_mul(C.t[b], cbnx));
#pragma unroll 1
    for (int a = 0; a < Q_FAR; ++a) {
      ff u[3];
      for (int d = 0; d < 3; ++d) u[d] = ff_add(F.w0[d], ff_mul(C.s[a], qb[d]));
      const ff unx = ff_add(w0nx, ff_mul(C.s[a], qnx));
      const ff eu = ff_dot3(ef, u);
      const ff Delta = ff_sub(ff_dot3(u, u), ff{2.f * eu.h, 2.f * eu.l});
      const ff r = ff_sqrt(ff_add(rho2, Delta));
      const ff delta = ff_div(Delta, ff_add(rho, r));
      const ffc ep = expi_ff(ff_mul(kf, delta), m, C);
      const ffc E = ffc_mul(Eref, ep);
      const ff ir = ff_rcp(r);
      const ff ir2 = ff_mul(ir, ir);
      const ff ir3 = ff_mul(ir2, ir);
      const ff ir5 = ff_mul(ir3, ir2);
      const ff kr = ff_mul(kf, r);
      const ff dnx = ff_sub(enx, unx);
      // a = e^{ikr}(1 - ikr), b = e^{ikr}(3 - (kr)^2 - 3ikr)
      const ff are = ff_add(E.re, ff_mul(E.im, kr));
      const ff aim = ff_sub(E.im, ff_mul(E.re, kr));
      const ff t3 = ff_sub(ff_make(3.f), ff_mul(kr, kr));
      const ff kr3 = ff_mul_f(kr, 3.f);
      const ff bre = ff_add(ff_mul(E.re, t3), ff_mul(E.im, kr3));
      const ff bim = ff_sub(ff_mul(E.im, t3), ff_mul(E.re, kr3));
      const ff wgt = ff_mul(F.two_area, C.W[a * Q_FAR + b]);
      const ff wir3 = ff_mul(wgt, ir3);
      const ff f = ff_mul(wir3, Cd);
      const ff g1 = ff_mul(wir3, Cg1);
      const ff g2 = ff_mul(ff_mul(ff_mul(wgt, ir5), dnx), Cd);
      Dre = ff_add(Dre, ff_mul(are, f));
      Dim = ff_add(Dim, ff_mul(aim, f));
      Hre = ff_add(Hre, ff_sub(ff_mul(are, g1), ff_mul(bre, g2)));
      Him = ff_add(Him, ff_sub(ff_mul(aim, g1), ff_mul(bim, g2)));
      if (SK) {
        // G = e^{ikr}/(4 pi r),  dG/dn_x = -a ((x-y).n_x)/(4 pi r^3)
        const ff gs = ff_mul(ff_mul(wgt, ir), C.inv4pi);
        Sre = ff_add(Sre, ff_mul(E.re, gs));
        Sim = ff_add(Sim, ff_mul(E.im, gs));
        const ff gk = ff_mul(ff_mul(wir3, dnx), C.inv4pi);
        Kre = ff_sub(Kre, ff_mul(are, gk));
        Kim = ff_sub(Kim, ff_mul(aim, gk));
      }
    }
  }
  acc[0] = Dre;
  acc[1] = Dim;
  acc[2] = Hre;
  acc[3] = Him;
  acc[4] = Sre;
  acc[5] = Sim;
  acc[6] = Kre;
  acc[7] = Kim;
}

template <bool SK>
__device__ void far_dh_ff(const FfElem& F, const ff ef[3], double dist, const ff nxf[3], double k, ff kf,
                          const FfConst& C, cd& D, cd& H, cd& S, cd& K) {
  ff a[8];
  far_sums_ff<SK>(F, ef, dist, nxf, k, kf, C, a);
  D = mkc(ff_to_d(a[0]), ff_to_d(a[1]));
  H = mkc(ff_to_d(a[2]), ff_to_d(a[3]));
  if (SK) {
    S = mkc(ff_to_d(a[4]), ff_to_d(a[5]));
    K = mkc(ff_to_d(a[6]), ff_to_d(a[7]));
  }
}

// D, H (S, K) by class: the far class through far_dh_ff, the near classes in FP64.
template <bool SK>
__device__ void element_dh_mixed(const Elem& E, const FfElem& F, const double shift[3], const ff shf[3],
                                 const double x[3], const ff xf[3], const double nx[3], const ff nxf[3], double k,
                                 ff kf, const QuadRules& qr, const FfConst& C, cd& D, cd& H, cd& S, cd& K) {
  double dc[3];
  for (int d = 0; d < 3; ++d) dc[d] = x[d] - (E.c[d] + shift[d]);
  const double r2 = dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2];
  const double dist = sqrt(r2);
  if (dist >= FAR_RATIO * E.hmax) {
    const ff ef[3] = {ff_sub(ff_sub(xf[0], F.c[0]), shf[0]), ff_sub(ff_sub(xf[1], F.c[1]), shf[1]),
                      ff_sub(ff_sub(xf[2], F.c[2]), shf[2])};
    far_dh_ff<SK>(F, ef, dist, nxf, k, kf, C, D, H, S, K);
    return;
  }
  if (SK)
    element_dhsk(E, shift, x, nx, k, qr, D, H, S, K);
  else
    element_dh(E, shift, x, nx, k, qr, D, H);
}

// The block entry T (Burton-Miller combination of D and H, with SK the
// admittance terms) of element E seen from x, dist = |x - (c + shift)| in
// FP64 as the caller computed it, rk = 1 / k.  The far class forms the
// rigid combination -(D + (i/k) H) in float-float and converts once; the
// near classes and the admittance combination run in FP64.
template <bool SK>
__device__ cd element_entry_mixed(const Elem& E, const FfElem& F, const double shift[3], const ff shf[3],
                                  const double x[3], const ff xf[3], const double nx[3], const ff nxf[3],
                                  double dist, double k, ff kf, double rk, ff rkf, cd beta, const QuadRules& qr,
                                  const FfConst& C) {
  cd D, H, S, K;
  if (dist >= FAR_RATIO * E.hmax) {
    const ff ef[3] = {ff_sub(ff_sub(xf[0], F.c[0]), shf[0]), ff_sub(ff_sub(xf[1], F.c[1]), shf[1]),
                      ff_sub(ff_sub(xf[2], F.c[2]), shf[2])};
    ff a[8];
    far_sums_ff<SK>(F, ef, dist, nxf, k, kf, C, a);
    if (!SK) {
      const ff tre = ff_sub(ff_mul(a[3], rkf), a[0]);        // -Re D + Im H / k
      const ff tim = ff_neg(ff_add(a[1], ff_mul(a[2], rkf)));  // -(Im D + Re H / k)
      return mkc(ff_to_d(tre), ff_to_d(tim));
    }
    D = mkc(ff_to_d(a[0]), ff_to_d(a[1]));
    H = mkc(ff_to_d(a[2]), ff_to_d(a[3]));
    S = mkc(ff_to_d(a[4]), ff_to_d(a[5]));
    K = mkc(ff_to_d(a[6]), ff_to_d(a[7]));
    return bm_entry_adm_rk(D, H, S, K, k, rk, beta);
  }
  if (SK) {
    element_dhsk(E, shift, x, nx, k, qr, D, H, S, K);
    return bm_entry_adm_rk(D, H, S, K, k, rk, beta);
  }
  element_dh(E, shift, x, nx, k, qr, D, H);
  return bm_entry_rk(D, H, rk);
}

// One thread per entry (o, i, j) of n_off blocks of n x n; block o goes to
// out + dest[o] * n * n.  The diagonal of the zero offset is left to
// k_self_terms.  Far-class entries are computed here; near and very-near
// entries (a fraction of a per cent) are appended to near_list for
// k_near_entries, which gives each of them a whole warp, or computed here
// when the list is full.
template <bool SK>
__global__ void k_build_blocks(const Elem* __restrict__ tel, const FfElem* __restrict__ tfel,
                               const Elem* __restrict__ el, const FfElem* __restrict__ fel, int n,
                               const double* __restrict__ shifts, const ff* __restrict__ shiftf,
                               const int64_t* __restrict__ dest, int n_off,
                               int zero_off, cd* __restrict__ out, double k, cd beta, BlockWrite bw, QuadRules qr,
                               FfConst C, unsigned long long* __restrict__ near_list,
                               unsigned long long* __restrict__ near_count, unsigned long long near_cap) {
  const ff kf = ff_from_d(k);
  const double rk = 1.0 / k;
  const ff rkf = ff_from_d(rk);
  const size_t nn = (size_t)n * n;
  const size_t total = nn * (size_t)n_off;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx / nn);
    const size_t rem = idx - (size_t)o * nn;
    const int i = (int)(rem / n);
    const int j = (int)(rem - (size_t)i * n);
    if (o == zero_off && i == j) continue;
    const Elem& Ti = tel[i];
    double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    // the target normal in float-float is the element's own (prepared once)
    const FfElem& Fi = tfel[i];
    const ff nxf[3] = {Fi.ny[0], Fi.ny[1], Fi.ny[2]};
    const ff xf[3] = {Fi.c[0], Fi.c[1], Fi.c[2]};
    double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const ff shf[3] = {shiftf[3 * o], shiftf[3 * o + 1], shiftf[3 * o + 2]};
    const Elem& Ej = el[j];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (Ej.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    if (dist < FAR_RATIO * Ej.hmax && near_list) {
      const unsigned long long slot = atomicAdd(near_count, 1ull);
      if (slot < near_cap) {
        near_list[slot] = idx;
        continue;
      }
    }
    bw.put(out + (size_t)dest[o] * nn + rem,
           element_entry_mixed<SK>(Ej, fel[j], sh, shf, x, xf, nx, nxf, dist, k, kf, rk, rkf, beta, qr, C));
  }
}

// Near and very-near entries listed by k_build_blocks, one warp per entry:
// the lanes share the 64 points of the 8 x 8 collapsed rule (near) or the
// 256 points of the rule on the four midpoint children (very near), in FP64,
// and the sums are reduced across the warp in a fixed order.
template <bool SK>
__global__ void __launch_bounds__(256) k_near_entries(const Elem* __restrict__ tel, const Elem* __restrict__ el, int n,
                                                      const double* __restrict__ shifts,
                                                      const int64_t* __restrict__ dest,
                                                      const unsigned long long* __restrict__ list,
                                                      const unsigned long long* __restrict__ count,
                                                      unsigned long long cap, cd* __restrict__ out, double k,
                                                      cd beta, BlockWrite bw, QuadRules qr) {
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
    const Elem& Ti = tel[i];
    const Elem& E = el[j];
    const double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    const double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    double v[3][3];
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) v[a][d] = E.v[a][d] + sh[d];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (E.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    const bool very = dist < NEAR_RATIO * E.hmax;
    const int npts = very ? 4 * Q_NEAR * Q_NEAR : Q_NEAR * Q_NEAR;
    cd D = mkc(0.0, 0.0), H = mkc(0.0, 0.0), S = mkc(0.0, 0.0), K = mkc(0.0, 0.0);
    for (int p = lane; p < npts; p += 32) {
      const int child = p / (Q_NEAR * Q_NEAR), q = p - child * Q_NEAR * Q_NEAR;
      const int ia = q / Q_NEAR, ib = q - ia * Q_NEAR;
      // triangle (A, Bv, Cv): the element, or child `child` in the order
      // (v0, m01, m20), (m01, v1, m12), (m20, m12, v2), (m01, m12, m20)
      double A[3], Bv[3], Cv[3], two_area = 2.0 * E.area;
      for (int d = 0; d < 3; ++d) {
        const double m01 = 0.5 * (v[0][d] + v[1][d]), m12 = 0.5 * (v[1][d] + v[2][d]),
                     m20 = 0.5 * (v[2][d] + v[0][d]);
        if (!very) {
          A[d] = v[0][d];
          Bv[d] = v[1][d];
          Cv[d] = v[2][d];
        } else if (child == 0) {
          A[d] = v[0][d];
          Bv[d] = m01;
          Cv[d] = m20;
        } else if (child == 1) {
          A[d] = m01;
          Bv[d] = v[1][d];
          Cv[d] = m12;
        } else if (child == 2) {
          A[d] = m20;
          Bv[d] = m12;
          Cv[d] = v[2][d];
        } else {
          A[d] = m01;
          Bv[d] = m12;
          Cv[d] = m20;
        }
      }
      if (very) two_area *= 0.25;
      const double sv = qr.t8[ia], tv = qr.t8[ib];
      double y[3];
      for (int d = 0; d < 3; ++d) y[d] = A[d] + sv * ((Bv[d] - A[d]) + tv * (Cv[d] - Bv[d]));
      kernel_point4<SK>(x, nx, y, E.nrm, two_area * sv * qr.w8[ia] * qr.w8[ib], k, D, H, S, K);
    }
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
    if (lane == 0) bw.put(out + (size_t)dest[o] * nn + rem, SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k));
  }
}

// Listed entries (o, i, j) of n_off blocks (idx = (o n + i) n + j), written
// to out[e]: the exact entries a multilevel near field keeps (its P2P pairs).
// Same classes and arithmetic as k_build_blocks; near and very-near entries
// in FP64 in the thread itself.  The self entry of the zero offset is left
// to k_self_terms.
template <bool SK>
__global__ void k_build_entries(const Elem* __restrict__ el, const FfElem* __restrict__ fel, int n,
                                const double* __restrict__ shifts, const ff* __restrict__ shiftf, int zero_off,
                                const int64_t* __restrict__ list, int64_t count, cd* __restrict__ out, double k,
                                cd beta, QuadRules qr, FfConst C) {
  const ff kf = ff_from_d(k);
  const size_t nn = (size_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const size_t idx = (size_t)list[e];
    const int o = (int)(idx / nn);
    const size_t rem = idx - (size_t)o * nn;
    const int i = (int)(rem / n);
    const int j = (int)(rem - (size_t)i * n);
    if (o == zero_off && i == j) continue;
    const Elem& Ti = el[i];
    double x[3] = {Ti.c[0], Ti.c[1], Ti.c[2]};
    double nx[3] = {Ti.nrm[0], Ti.nrm[1], Ti.nrm[2]};
    const FfElem& Fi = fel[i];
    const ff nxf[3] = {Fi.ny[0], Fi.ny[1], Fi.ny[2]};
    const ff xf[3] = {Fi.c[0], Fi.c[1], Fi.c[2]};
    double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const ff shf[3] = {shiftf[3 * o], shiftf[3 * o + 1], shiftf[3 * o + 2]};
    cd D, H, S, K;
    element_dh_mixed<SK>(el[j], fel[j], sh, shf, x, xf, nx, nxf, k, kf, qr, C, D, H, S, K);
    out[e] = SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k);
  }
}

// sin x - x cos x without cancellation: series for |x| < 0.5.
__device__ double sin_minus_xcos(double x) {
  if (fabs(x) < 0.5) {
    double x2 = x * x, term = x * x2, acc = 0.0;
    // (-1)^{j+1} 2j x^{2j+1} / (2j+1)!
    double fact = 6.0;   // 3!
    for (int j = 1; j <= 9; ++j) {
      double c = ((j & 1) ? 1.0 : -1.0) * 2.0 * j / fact;
      acc += c * term;
      term *= x2;
      fact *= (double)(2 * j + 2) * (double)(2 * j + 3);
    }
    return acc;
  }
  double s, c;
  sincos(x, &s, &c);
  return s - x * c;
}

// Self term of element i (x_i at its centroid, on the flat panel):
// D_ii = 0, H_ii = (1/4pi)[fp int r^-3 + int (e^{ikr}(1-ikr) - 1) r^-3];
// with an admittance (beta != 0) also K_ii = 0 and
// S_ii = (1/4pi)[int 1/r + int (e^{ikr} - 1)/r], the 1/r part in closed form
// (polar coordinates about x: an edge at distance h with end coordinates
// t_a, t_b along it gives h ln((t_b + |b - x|)/(t_a + |a - x|))).
__global__ void k_self_terms(const Elem* __restrict__ el, int n, cd* __restrict__ block0, double k, cd beta,
                             QuadRules qr, const int64_t* __restrict__ slot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Elem& E = el[i];
  const double* x = E.c;
  const bool adm = beta.x != 0.0 || beta.y != 0.0;
  double fp = 0.0, invr = 0.0;
  for (int e = 0; e < 3; ++e) {
    const double* a = E.v[e];
    const double* b = E.v[(e + 1) % 3];
    double eh[3], am[3], bm[3];
    double L = 0.0;
    for (int d = 0; d < 3; ++d) {
      eh[d] = b[d] - a[d];
      L += eh[d] * eh[d];
      am[d] = a[d] - x[d];
      bm[d] = b[d] - x[d];
    }
    L = sqrt(L);
    for (int d = 0; d < 3; ++d) eh[d] /= L;
    double ta = am[0] * eh[0] + am[1] * eh[1] + am[2] * eh[2];
    double tb = bm[0] * eh[0] + bm[1] * eh[1] + bm[2] * eh[2];
    double hv[3] = {am[0] - ta * eh[0], am[1] - ta * eh[1], am[2] - ta * eh[2]};
    double he = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
    double ra = sqrt(am[0] * am[0] + am[1] * am[1] + am[2] * am[2]);
    double rb = sqrt(bm[0] * bm[0] + bm[1] * bm[1] + bm[2] * bm[2]);
    fp -= (tb / rb - ta / ra) / he;
    invr += he * log((tb + rb) / (ta + ra));
  }
  double rem_re = 0.0, rem_im = 0.0, srem_re = 0.0, srem_im = 0.0;
  for (int e = 0; e < 3; ++e) {
    const double* a = E.v[e];
    const double* b = E.v[(e + 1) % 3];
    double ax[3], ba[3], cr[3];
    for (int d = 0; d < 3; ++d) {
      ax[d] = a[d] - x[d];
      ba[d] = b[d] - a[d];
    }
    double bx[3] = {b[0] - x[0], b[1] - x[1], b[2] - x[2]};
    cr[0] = ax[1] * bx[2] - ax[2] * bx[1];
    cr[1] = ax[2] * bx[0] - ax[0] * bx[2];
    cr[2] = ax[0] * bx[1] - ax[1] * bx[0];
    const double two_area = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int p = 0; p < Q_SELF; ++p) {
      const double s = qr.t8[p];
      const double ws = two_area * s * qr.w8[p];
      for (int q = 0; q < Q_SELF; ++q) {
        double y[3];
        for (int d = 0; d < 3; ++d) y[d] = x[d] + s * (ax[d] + qr.t8[q] * ba[d]);
        double dx = y[0] - x[0], dy = y[1] - x[1], dz = y[2] - x[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double kr = k * r;
        double sh = sin(0.5 * kr);
        const double skr = sin(kr);
        double re = -2.0 * sh * sh + kr * skr;       // cos kr + kr sin kr - 1
        double im = sin_minus_xcos(kr);              // sin kr - kr cos kr
        double wr = ws * qr.w8[q] / (r * r * r);
        rem_re += wr * re;
        rem_im += wr * im;
        if (adm) {
          const double w1 = ws * qr.w8[q] / r;       // (e^{ikr} - 1)/r
          srem_re += w1 * (-2.0 * sh * sh);
          srem_im += w1 * skr;
        }
      }
    }
  }
  const double inv4pi = 0.25 / PI;
  cd H = mkc((fp + rem_re) * inv4pi, rem_im * inv4pi);
  // 1/2 - (i/k) H
  cd t = mkc(0.5 + H.y / k, -H.x / k);
  if (adm) {
    // + beta (1/2 - i k S)
    const cd S = mkc((invr + srem_re) * inv4pi, srem_im * inv4pi);
    t = cadd(t, cmul(beta, mkc(0.5 + k * S.y, -k * S.x)));
  }
  if (slot) {
    if (slot[i] >= 0) block0[slot[i]] = t;   // listed entries: the slot of (i, i)
  } else {
    block0[(size_t)i * n + i] = t;
  }
}

// ------------------------------------------------------- right-hand side --
// p_inc and dp_inc/dn at x (normal nrm) of one incident field: a plane wave
// amp e^{ik d.x} (Eq. (planewave)) or a monopole amp e^{ikr}/r, r = |x - x_s|.
__device__ void incident_free(const IncDev& in, const double x[3], const double nrm[3], double k, cd& p, cd& dp) {
  if (in.kind == 0) {
    double ph = 0.0, dn = 0.0;
    for (int d = 0; d < 3; ++d) {
      ph += in.v[d] * x[d];
      dn += in.v[d] * nrm[d];
    }
    double s, c;
    sincos(k * ph, &s, &c);
    p = cmul(in.amp, mkc(c, s));
    dp = cmul(mkc(0.0, k * dn), p);   // i k (d.n) p
    return;
  }
  double rv[3], r2 = 0.0, rn = 0.0;
  for (int d = 0; d < 3; ++d) {
    rv[d] = x[d] - in.v[d];
    r2 += rv[d] * rv[d];
    rn += rv[d] * nrm[d];
  }
  const double r = sqrt(r2);
  double s, c;
  sincos(k * r, &s, &c);
  p = cmulr(cmul(in.amp, mkc(c, s)), 1.0 / r);
  // d/dn e^{ikr}/r = e^{ikr}/r (ikr - 1)/r (r_vec . n)/r
  dp = cmul(p, mkc(-rn / r2, k * rn / r));
}

// With a plane, the image R_p p_inc(M x): its normal derivative along n is the
// derivative of p_inc at M x along R n.
__device__ void incident_at(const IncDev& in, const PlaneDev& pl, const double x[3], const double nrm[3], double k,
                            cd& p, cd& dp) {
  incident_free(in, x, nrm, k, p, dp);
  if (pl.on) {
    double xm[3], nm[3];
    for (int d = 0; d < 3; ++d) {
      xm[d] = x[d];
      nm[d] = nrm[d];
    }
    xm[pl.axis] = 2.0 * pl.offset - x[pl.axis];
    nm[pl.axis] = -nrm[pl.axis];
    cd pi, dpi;
    incident_free(in, xm, nm, k, pi, dpi);
    p = cfma(pl.Rp, pi, p);
    dp = cfma(pl.Rp, dpi, dp);
  }
}

// b_r(x_i) = p_inc(x_i) + (i/k) dp_inc/dn(x_i) at every collocation point.
__global__ void k_rhs_incident(const Elem* __restrict__ el, int n, CellGrid g, double k, int R,
                               const IncDev* __restrict__ inc, PlaneDev pl, cd* __restrict__ b) {
  const size_t N = (size_t)n * g.ncells;
  const size_t total = N * R;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / N);
    const size_t gi = idx - (size_t)r * N;
    const int c = (int)(gi / n);
    const int i = (int)(gi - (size_t)c * n);
    double x[3];
    g.cell_position(c, x);
    const Elem& E = el[i];
    for (int d = 0; d < 3; ++d) x[d] += E.c[d];
    cd p, dp;
    incident_at(inc[r], pl, x, E.nrm, k, p, dp);
    b[idx] = mkc(p.x - dp.y / k, p.y + dp.x / k);   // p + (i/k) dp
  }
}

// ---------------------------------------------------------- field points --
// out[r][p] = p_inc,r(x_p) + sum_{c, j} (D + i k beta S)(x_p, E_j + pos_c) surf[r][c*n + j]
// (Eq. (cbie) with c = 1; with an admittance the single layer of
// dp/dn_m = -i k beta p joins the double layer), and for a half-space
// operator R_p times the same sum over the mirrored elements: refl holds the
// reflected unit cell (R v, reversed winding), placed for cell c at
// R pos_c + 2 offset e.
__global__ void __launch_bounds__(256) k_field(const Elem* __restrict__ el, const Elem* __restrict__ refl, int n,
                                               CellGrid g, double k, cd beta, PlaneDev pl, int R,
                                               const IncDev* __restrict__ inc, const cd* __restrict__ surf,
                                               int64_t npts, const double* __restrict__ pts, cd* __restrict__ out,
                                               QuadRules qr) {
  // one CTA per (rhs, point): the threads split the elements of every cell
  // (and their images) and the partial sums are reduced in a fixed order
  __shared__ double sre[256], sim[256];
  const bool adm = beta.x != 0.0 || beta.y != 0.0;
  const cd ikb = mkc(-k * beta.y, k * beta.x);
  const int64_t total = (int64_t)npts * R;
  const size_t N = (size_t)n * g.ncells;
  const int64_t items = (int64_t)g.ncells * n;
  for (int64_t idx = blockIdx.x; idx < total; idx += gridDim.x) {
    const int r = (int)(idx / npts);
    const int64_t p = idx - (int64_t)r * npts;
    double x[3] = {pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]};
    double nx[3] = {0.0, 0.0, 1.0};
    cd part = mkc(0.0, 0.0);
    for (int64_t it = threadIdx.x; it < items; it += blockDim.x) {
      const int c = (int)(it / n), j = (int)(it - (int64_t)c * n);
      const cd pj = surf[(size_t)r * N + (size_t)c * n + j];
      double pos[3];
      g.cell_position(c, pos);
      for (int side = 0; side < (pl.on ? 2 : 1); ++side) {
        const Elem* els = side ? refl : el;
        if (side) pos[pl.axis] = 2.0 * pl.offset - pos[pl.axis];
        cd D, H, S, K;
        if (adm) {
          element_dhsk(els[j], pos, x, nx, k, qr, D, H, S, K);
          D = cfma(ikb, S, D);
        } else {
          element_dh(els[j], pos, x, nx, k, qr, D, H);
        }
        const cd v = cmul(D, pj);
        part = side ? cfma(pl.Rp, v, part) : cadd(part, v);
      }
    }
    sre[threadIdx.x] = part.x;
    sim[threadIdx.x] = part.y;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        sre[threadIdx.x] += sre[threadIdx.x + s];
        sim[threadIdx.x] += sim[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      cd acc, dummy;
      incident_at(inc[r], pl, x, nx, k, acc, dummy);
      out[idx] = cadd(acc, mkc(sre[0], sim[0]));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------- insertion loss --
// Incident field alone at the points (with its image for a half-space
// operator), out[r][p].
__global__ void k_incident_points(const IncDev* __restrict__ inc, PlaneDev pl, double k, int R, int64_t npts,
                                  const double* __restrict__ pts, cd* __restrict__ out) {
  const int64_t total = (int64_t)npts * R;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / npts);
    const int64_t p = idx - (int64_t)r * npts;
    const double x[3] = {pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]};
    const double nx[3] = {0.0, 0.0, 1.0};
    cd v, dv;
    incident_at(inc[r], pl, x, nx, k, v, dv);
    out[idx] = v;
  }
}

// sums[0] = sum_p |sum_r inc[r][p]|, sums[1] = sum_p |sum_r tot[r][p]| in one
// CTA (fixed order: deterministic).
__global__ void k_il_sums(const cd* __restrict__ inc, const cd* __restrict__ tot, int R, int64_t npts,
                          double* __restrict__ sums) {
  __shared__ double a[256], b[256];
  double sa = 0.0, sb = 0.0;
  for (int64_t p = threadIdx.x; p < npts; p += blockDim.x) {
    cd ci = mkc(0.0, 0.0), ct = mkc(0.0, 0.0);
    for (int r = 0; r < R; ++r) {
      ci = cadd(ci, inc[(int64_t)r * npts + p]);
      ct = cadd(ct, tot[(int64_t)r * npts + p]);
    }
    sa += hypot(ci.x, ci.y);
    sb += hypot(ct.x, ct.y);
  }
  a[threadIdx.x] = sa;
  b[threadIdx.x] = sb;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      a[threadIdx.x] += a[threadIdx.x + s];
      b[threadIdx.x] += b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] = a[0];
    sums[1] = b[0];
  }
}

// ------------------------------------------------------------ host side --
fmpb_status upload_mesh(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, DeviceMesh& m,
                        cudaStream_t st) {
  if (!verts || !tris || nv < 3 || ntri < 1 || ntri > (1 << 20)) {
    set_error("mesh: need verts (nv >= 3), tris (1 <= ntri <= 2^20)");
    return FMPB_EINVAL;
  }
  // host validation: indices in range, finite coordinates, non-degenerate triangles
  for (int64_t e = 0; e < 3 * nv; ++e)
    if (!std::isfinite(verts[e])) {
      set_error("mesh: vertex coordinate %lld is not finite", (long long)e);
      return FMPB_EMESH;
    }
  for (int64_t t = 0; t < ntri; ++t) {
    const int32_t* tv = tris + 3 * t;
    for (int a = 0; a < 3; ++a)
      if (tv[a] < 0 || tv[a] >= nv) {
        set_error("mesh: triangle %lld references vertex %d (nv = %lld)", (long long)t, tv[a], (long long)nv);
        return FMPB_EMESH;
      }
    const double* a = verts + 3 * tv[0];
    const double* b = verts + 3 * tv[1];
    const double* c = verts + 3 * tv[2];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    double l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    double ca = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
    if (!(ca > 1e-24 * l1 * l2)) {
      set_error("mesh: triangle %lld has (near) zero area", (long long)t);
      return FMPB_EMESH;
    }
  }
  m.n = (int)ntri;
  double* dverts = nullptr;
  int32_t* dtris = nullptr;
  FMPB_CUDA(cudaMalloc(&dverts, sizeof(double) * 3 * nv));
  cudaError_t e = cudaMalloc(&dtris, sizeof(int32_t) * 3 * ntri);
  if (e == cudaSuccess) e = cudaMalloc(&m.el, sizeof(Elem) * ntri);
  if (e == cudaSuccess) e = cudaMalloc(&m.qr_dev, sizeof(QuadRules));
  if (e == cudaSuccess) e = cudaMalloc(&m.ffel, sizeof(FfElem) * ntri);
  if (e == cudaSuccess) e = cudaMalloc(&m.fc_dev, sizeof(FfConst));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dverts, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dtris, tris, sizeof(int32_t) * 3 * ntri, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    FMPB_LAUNCH("prepare_elements", st, k_prepare_elements<<<grid_for(ntri, 128), 128, 0, st>>>(dverts, dtris, (int)ntri, m.el));
    FMPB_LAUNCH("gauss_legendre", st, k_gauss_legendre<<<1, 32, 0, st>>>(m.qr_dev));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    FMPB_LAUNCH("prepare_ff", st, k_prepare_ff<<<grid_for(ntri, 128), 128, 0, st>>>(m.el, (int)ntri, m.ffel, m.qr_dev, m.fc_dev));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&m.qr, m.qr_dev, sizeof(QuadRules), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&m.fc, m.fc_dev, sizeof(FfConst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dverts);
  cudaFree(dtris);
  if (e != cudaSuccess) return cuda_status(e, "upload_mesh");
  // cell radius about the origin (expansion centre), from the host copy
  double rho = 0.0;
  for (int64_t t = 0; t < ntri; ++t)
    for (int a = 0; a < 3; ++a) {
      const double* v = verts + 3 * tris[3 * t + a];
      rho = fmax(rho, sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
  m.radius = rho;
  return FMPB_OK;
}

void free_mesh(DeviceMesh& m) {
  if (m.el) cudaFree(m.el);
  if (m.qr_dev) cudaFree(m.qr_dev);
  if (m.ffel) cudaFree(m.ffel);
  if (m.fc_dev) cudaFree(m.fc_dev);
  if (m.q9) cudaFree(m.q9);
  if (m.q9_far) cudaFree(m.q9_far);
  if (m.q9_farff) cudaFree(m.q9_farff);
  if (m.q9_near) cudaFree(m.q9_near);
  m.el = nullptr;
  m.qr_dev = nullptr;
  m.ffel = nullptr;
  m.fc_dev = nullptr;
  m.q9 = nullptr;
  m.q9_far = nullptr;
  m.q9_farff = nullptr;
  m.q9_near = nullptr;
}

fmpb_status build_blocks(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                         const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st,
                         const ImageBlocks* img) {
  if (m.nodes == 9) {
    if (img) return build_blocks_q9p(m, g, k, beta, n_off, offsets, dest_host, out, st, img);
    return build_blocks_q9(m, g, k, beta, n_off, offsets, dest_host, out, st);
  }
  // shifts: -delta . lattice, or the image shifts given by the caller
  std::vector<double> shifts(3 * (size_t)n_off);
  int zero_off = -1;
  for (int o = 0; o < n_off; ++o) {
    const int32_t* dl = offsets + 3 * o;
    if (!img && dl[0] == 0 && dl[1] == 0 && dl[2] == 0) zero_off = o;
    for (int d = 0; d < 3; ++d)
      shifts[3 * o + d] = img ? img->shifts[3 * o + d]
                              : -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
  }
  BlockWrite bw{mkc(1.0, 0.0), 0, 0};
  if (img) bw = BlockWrite{img->scale, 1, img->accumulate ? 1 : 0};
  // collocation points from m, elements from the reflected cell for images
  const DeviceMesh& src = img ? *img->source : m;
  if (src.n != m.n) {
    set_error("build_blocks: source and target cells differ in size");
    return FMPB_EINVAL;
  }
  // the same shifts as float-float pairs (hi = nearest float, lo = nearest float of the rest)
  std::vector<ff> shiftf(3 * (size_t)n_off);
  for (size_t q = 0; q < shiftf.size(); ++q) {
    const float hi = (float)shifts[q];
    shiftf[q] = ff{hi, (float)(shifts[q] - (double)hi)};
  }
  double* dshift = nullptr;
  ff* dshiftf = nullptr;
  int64_t* ddest = nullptr;
  FMPB_CUDA(cudaMalloc(&dshift, sizeof(double) * 3 * n_off));
  cudaError_t e = cudaMalloc(&ddest, sizeof(int64_t) * n_off);
  if (e == cudaSuccess) e = cudaMalloc(&dshiftf, sizeof(ff) * 3 * n_off);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dshift, shifts.data(), sizeof(double) * 3 * n_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dshiftf, shiftf.data(), sizeof(ff) * 3 * n_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ddest, dest_host, sizeof(int64_t) * n_off, cudaMemcpyHostToDevice, st);
  // list of near and very-near entries for k_near_entries (entries beyond
  // its capacity are computed by k_build_blocks itself)
  const size_t total = (size_t)m.n * m.n * n_off;
  const unsigned long long near_cap = (unsigned long long)std::min<size_t>(total, (size_t)8 << 20);
  unsigned long long* near_list = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&near_list, sizeof(unsigned long long) * (near_cap + 1));
  unsigned long long* near_count = near_list ? near_list + near_cap : nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(near_count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    // short-lived CTAs (about a dozen entries per thread at the headline's
    // size): a build that runs beside a solve on a lower-priority stream
    // frees SM slots every few microseconds, so the solve's kernels do not
    // wait for CTAs that would otherwise hold their SMs for tens of ms
    unsigned blocks = (unsigned)std::min<size_t>(grid_for(total, 128), (size_t)152 * 1024);
    if (beta.x == 0.0 && beta.y == 0.0) {
      FMPB_LAUNCH("build_blocks", st, k_build_blocks<false><<<blocks, 128, 0, st>>>(m.el, m.ffel, src.el, src.ffel, m.n, dshift, dshiftf, ddest, n_off, zero_off, out, k, beta, bw, m.qr, m.fc, near_list, near_count, near_cap));
      FMPB_LAUNCH("build_near", st, k_near_entries<false><<<152 * 128, 256, 0, st>>>(m.el, src.el, m.n, dshift, ddest, near_list, near_count, near_cap, out, k, beta, bw, m.qr));
    } else {
      FMPB_LAUNCH("build_blocks_adm", st, k_build_blocks<true><<<blocks, 128, 0, st>>>(m.el, m.ffel, src.el, src.ffel, m.n, dshift, dshiftf, ddest, n_off, zero_off, out, k, beta, bw, m.qr, m.fc, near_list, near_count, near_cap));
      FMPB_LAUNCH("build_near_adm", st, k_near_entries<true><<<152 * 128, 256, 0, st>>>(m.el, src.el, m.n, dshift, ddest, near_list, near_count, near_cap, out, k, beta, bw, m.qr));
    }
    if (zero_off >= 0)
      FMPB_LAUNCH("self_terms", st, k_self_terms<<<grid_for(m.n, 64), 64, 0, st>>>(m.el, m.n, out + (size_t)dest_host[zero_off] * m.n * m.n,
                                                     k, beta, m.qr, nullptr));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dshift);
  cudaFree(dshiftf);
  cudaFree(ddest);
  cudaFree(near_list);
  if (e != cudaSuccess) return cuda_status(e, "build_blocks");
  return FMPB_OK;
}

fmpb_status build_entries(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                          const int32_t* offsets, const int64_t* list, int64_t count, const int64_t* self_slot,
                          cd* out, cudaStream_t st) {
  if (m.nodes == 9) return build_entries_q9(m, g, k, beta, n_off, offsets, list, count, self_slot, out, st);
  std::vector<double> shifts(3 * (size_t)n_off);
  int zero_off = -1;
  for (int o = 0; o < n_off; ++o) {
    const int32_t* dl = offsets + 3 * o;
    if (dl[0] == 0 && dl[1] == 0 && dl[2] == 0) zero_off = o;
    for (int d = 0; d < 3; ++d) shifts[3 * o + d] = -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
  }
  std::vector<ff> shiftf(3 * (size_t)n_off);
  for (size_t q = 0; q < shiftf.size(); ++q) {
    const float hi = (float)shifts[q];
    shiftf[q] = ff{hi, (float)(shifts[q] - (double)hi)};
  }
  double* dshift = nullptr;
  ff* dshiftf = nullptr;
  FMPB_CUDA(cudaMallocAsync(&dshift, sizeof(double) * 3 * n_off, st));
  FMPB_CUDA(cudaMallocAsync(&dshiftf, sizeof(ff) * 3 * n_off, st));
  FMPB_CUDA(cudaMemcpyAsync(dshift, shifts.data(), sizeof(double) * 3 * n_off, cudaMemcpyHostToDevice, st));
  FMPB_CUDA(cudaMemcpyAsync(dshiftf, shiftf.data(), sizeof(ff) * 3 * n_off, cudaMemcpyHostToDevice, st));
  if (count > 0) {
    const unsigned blocks = (unsigned)std::min<int64_t>((count + 127) / 128, 152 * 64);
    if (beta.x == 0.0 && beta.y == 0.0)
      FMPB_LAUNCH("build_entries", st, k_build_entries<false><<<blocks, 128, 0, st>>>(m.el, m.ffel, m.n, dshift, dshiftf, zero_off, list, count, out, k, beta, m.qr, m.fc));
    else
      FMPB_LAUNCH("build_entries_adm", st, k_build_entries<true><<<blocks, 128, 0, st>>>(m.el, m.ffel, m.n, dshift, dshiftf, zero_off, list, count, out, k, beta, m.qr, m.fc));
  }
  if (zero_off >= 0 && self_slot)
    FMPB_LAUNCH("self_terms", st, k_self_terms<<<grid_for(m.n, 64), 64, 0, st>>>(m.el, m.n, out, k, beta, m.qr, self_slot));
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaFreeAsync(dshift, st));
  FMPB_CUDA(cudaFreeAsync(dshiftf, st));
  return FMPB_OK;
}

static fmpb_status upload_incident(int R, const fmpb_incident* inc, double k, IncDev** out, cudaStream_t st) {
  std::vector<IncDev> h(R);
  for (int r = 0; r < R; ++r) {
    const fmpb_incident& a = inc[r];
    if (a.kind != FMPB_INC_PLANE && a.kind != FMPB_INC_MONOPOLE) {
      set_error("incident field %d: unknown kind %d", r, a.kind);
      return FMPB_EINVAL;
    }
    double nrm = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!std::isfinite(a.vec[d])) {
        set_error("incident field %d: vector not finite", r);
        return FMPB_EINVAL;
      }
      h[r].v[d] = a.vec[d];
      nrm += a.vec[d] * a.vec[d];
    }
    if (a.kind == FMPB_INC_PLANE && !(fabs(nrm - 1.0) < 1e-6)) {
      set_error("rhs: direction %d is not a unit vector", r);
      return FMPB_EINVAL;
    }
    h[r].kind = a.kind;
    h[r].amp = mkc(a.amp.re, a.amp.im);
  }
  (void)k;
  IncDev* d = nullptr;
  FMPB_CUDA(cudaMallocAsync(&d, sizeof(IncDev) * R, st));
  FMPB_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(IncDev) * R, cudaMemcpyHostToDevice, st));
  *out = d;
  return FMPB_OK;
}

fmpb_status rhs_incident(const DeviceMesh& m, const CellGrid& g, double k, int R, const fmpb_incident* inc,
                         const PlaneDev& pl, cd* b, cudaStream_t st) {
  IncDev* dinc = nullptr;
  FMPB_TRY(upload_incident(R, inc, k, &dinc, st));
  const size_t total = (size_t)m.n * g.ncells * R;
  FMPB_LAUNCH("rhs_incident", st, k_rhs_incident<<<std::min<size_t>(grid_for(total, 256), 152 * 32), 256, 0, st>>>(m.el, m.n, g, k, R, dinc, pl, b));
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaFreeAsync(dinc, st));
  return FMPB_OK;
}

fmpb_status field_incident(const DeviceMesh& m, const DeviceMesh* refl, const CellGrid& g, double k, cd beta,
                           const PlaneDev& pl, int R, const cd* surf, const fmpb_incident* inc, int64_t npts,
                           const double* pts, cd* out, cudaStream_t st) {
  if (pl.on && !refl) {
    set_error("field: half-space operator without its reflected cell");
    return FMPB_EINVAL;
  }
  if (m.nodes == 9) {
    // nine-node quadrilaterals: the incident field (with its image), then the
    // scattered part added
    IncDev* dq = nullptr;
    FMPB_TRY(upload_incident(R, inc, k, &dq, st));
    const int64_t tq = (int64_t)npts * R;
    FMPB_LAUNCH("incident_points", st, k_incident_points<<<(unsigned)std::min<int64_t>((tq + 255) / 256, 152 * 32), 256, 0, st>>>(dq, pl, k, R, npts, pts, out));
    FMPB_CUDA(cudaGetLastError());
    FMPB_TRY(field_scattered_q9(m, refl, pl, g, k, beta, R, surf, npts, pts, out, st));
    FMPB_CUDA(cudaFreeAsync(dq, st));
    return FMPB_OK;
  }
  IncDev* dinc = nullptr;
  FMPB_TRY(upload_incident(R, inc, k, &dinc, st));
  const size_t total = (size_t)npts * R;
  FMPB_LAUNCH("field", st, k_field<<<(unsigned)std::min<size_t>(total, 152 * 16), 256, 0, st>>>(m.el, pl.on ? refl->el : m.el, m.n, g, k, beta, pl, R, dinc, surf, npts, pts, out, m.qr));
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaFreeAsync(dinc, st));
  return FMPB_OK;
}

fmpb_status insertion_loss(const DeviceMesh& m, const DeviceMesh* refl, const CellGrid& g, double k, cd beta,
                           const PlaneDev& pl, int R, const cd* surf, const fmpb_incident* inc, int64_t npts,
                           const double* pts, double* il, cudaStream_t st) {
  cd* tot = nullptr;
  cd* incv = nullptr;
  double* sums = nullptr;
  FMPB_CUDA(cudaMallocAsync(&tot, sizeof(cd) * (size_t)R * npts, st));
  FMPB_CUDA(cudaMallocAsync(&incv, sizeof(cd) * (size_t)R * npts, st));
  FMPB_CUDA(cudaMallocAsync(&sums, sizeof(double) * 2, st));
  FMPB_TRY(field_incident(m, refl, g, k, beta, pl, R, surf, inc, npts, pts, tot, st));
  IncDev* dinc = nullptr;
  FMPB_TRY(upload_incident(R, inc, k, &dinc, st));
  const int64_t total = (int64_t)npts * R;
  FMPB_LAUNCH("incident_points", st, k_incident_points<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(dinc, pl, k, R, npts, pts, incv));
  FMPB_LAUNCH("il_sums", st, k_il_sums<<<1, 256, 0, st>>>(incv, tot, R, npts, sums));
  FMPB_CUDA(cudaGetLastError());
  double h[2] = {0.0, 0.0};
  FMPB_CUDA(cudaMemcpyAsync(h, sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaFreeAsync(dinc, st));
  FMPB_CUDA(cudaFreeAsync(tot, st));
  FMPB_CUDA(cudaFreeAsync(incv, st));
  FMPB_CUDA(cudaFreeAsync(sums, st));
  FMPB_CUDA(cudaStreamSynchronize(st));
  if (!(h[1] > 0.0)) {
    set_error("insertion_loss: the total field vanishes at every point");
    return FMPB_EINVAL;
  }
  *il = 20.0 * log10(h[0] / h[1]);
  return FMPB_OK;
}

}  // namespace fmpb

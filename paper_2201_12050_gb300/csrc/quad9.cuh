// Nine-node quadratic quadrilaterals (the element family of Sec. 2.1 and
// Eq. (matrixBEM)) with one constant pressure per element, collocated at the
// element centre y(0, 0): geometry, the regular class rules and the singular
// self terms.  Host-and-device code: the kernels of quad9.cu call these
// functions, and the host uses them to validate a mesh.
//
// Element.  y(xi, eta) = sum_a N_a(xi, eta) Y_a on [-1, 1]^2 with N_a the
// products of the 1-D quadratic Lagrange polynomials on -1, 0, 1 (node (i, j)
// at 3 j + i, i along xi).  Written in monomials about the centre,
//   y(xi, eta) = sum_{p,q = 0..2} a_pq xi^p eta^q,
// exactly (the map is biquadratic): y(0, 0) = a_00 = Y_4, y_xi = a_10,
// y_eta = a_01, y_xixi = 2 a_20, y_xieta = a_11, y_etaeta = 2 a_02.  The
// self terms form y - x from these coefficients, so that the small
// differences near the collocation point carry no cancellation.
//
// Regular classes (d = |x - y(0, 0)|, h = longest corner-to-corner chord,
// thresholds of the triangle rule): far d >= 4 h: 4 x 4 Gauss-Legendre;
// near 1.5 h <= d < 4 h: 8 x 8; very near: 8 x 8 on each parameter quarter.
//
// Self term (polar coordinates (rho, theta) about (0, 0) in the parameter
// plane; the square split into four triangles with apex at the centre;
// 16-point Gauss-Legendre in theta on each side's range and in rho on
// [0, rho_hat(theta)]): D, S, K directly (weakly singular on the curved
// element), H as the Hadamard finite part with a spherical exclusion.  With
// y - x = rho A + rho^2 B + O(rho^3), beta = |A| and |J| = J0 + rho J1 +
// O(rho^2), F = H |J| rho = F_-2 / rho^2 + F_-1 / rho + O(1),
//   F_-2 = J0 / (4 pi beta^3),  F_-1 = (J1 - 3 J0 (A.B) / beta^2) / (4 pi beta^3),
// and the finite part is
//   int_theta int_0^rho_hat (F - F_-2/rho^2 - F_-1/rho) drho dtheta
//   + int_theta [F_-1 ln(rho_hat beta) + F_-2 ((A.B)/beta^2 - 1/rho_hat)] dtheta.
#pragma once
#include "common.cuh"

namespace fmpb {

constexpr int Q9_FAR = 16;         // points of the far rule
constexpr int Q9_NEAR = 64;        // points of the near rule
constexpr int Q9_VNEAR = 256;      // points of the very-near rule
constexpr int Q9_NEAR_TAB = Q9_NEAR + Q9_VNEAR;
constexpr int Q9_THETA = 64;       // angular nodes of the self rule (4 sides x 16)
constexpr int Q9_RHO = 16;         // radial nodes per angular node

// Gauss-Legendre nodes t (ascending) and weights w on [0, 1] (the 24-point
// rule serves the self terms of pressure of order 1 and 2).
struct Q9Rules {
  double t4[4], w4[4], t8[8], w8[8], t16[16], w16[16], t24[24], w24[24];
};

struct Q9Elem {
  double Y[9][3];   // nodes
  double c[3];      // y(0, 0): the collocation point
  double nrm[3];    // unit normal at the centre, into the fluid
  double hmax;      // longest chord between cyclically adjacent corners (nodes 0, 2, 8, 6)
  double area;      // surface area (4 x 4 rule)
};

// Monomial coefficients a_pq (index 3 q + p) of one element.
__host__ __device__ inline void q9_monomials(const double Y[9][3], double a[9][3]) {
  // L_0(t) = (t^2 - t)/2, L_1(t) = 1 - t^2, L_2(t) = (t^2 + t)/2: coefficient of t^p
  const double c[3][3] = {{0.0, -0.5, 0.5}, {1.0, 0.0, -1.0}, {0.0, 0.5, 0.5}};
  for (int q = 0; q < 3; ++q)
    for (int p = 0; p < 3; ++p)
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
          for (int i = 0; i < 3; ++i) s += c[i][p] * c[j][q] * Y[3 * j + i][d];
        a[3 * q + p][d] = s;
      }
}

// y, y_xi, y_eta at (xi, eta) from the monomial coefficients.
__host__ __device__ inline void q9_eval(const double a[9][3], double xi, double eta, double y[3], double yx[3],
                                        double ye[3]) {
  const double xp[3] = {1.0, xi, xi * xi}, ep[3] = {1.0, eta, eta * eta};
  for (int d = 0; d < 3; ++d) {
    double s = 0.0, sx = 0.0, se = 0.0;
    for (int q = 0; q < 3; ++q)
      for (int p = 0; p < 3; ++p) {
        const double ad = a[3 * q + p][d];
        s += ad * xp[p] * ep[q];
        if (p > 0) sx += p * ad * xp[p - 1] * ep[q];
        if (q > 0) se += q * ad * xp[p] * ep[q - 1];
      }
    y[d] = s;
    yx[d] = sx;
    ye[d] = se;
  }
}

__host__ __device__ inline void q9_cross(const double u[3], const double v[3], double w[3]) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}
__host__ __device__ inline double q9_dot(const double u[3], const double v[3]) {
  return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

// Parameter point and weight (on [-1, 1]^2) of point p of a class rule:
// cls 0: 4 x 4 (16 points), 1: 8 x 8 (64), 2: 8 x 8 on each quarter (256).
__host__ __device__ inline void q9_rule_point(const Q9Rules& R, int cls, int p, double* xi, double* eta,
                                              double* w) {
  if (cls == 0) {
    const int a = p / 4, b = p % 4;
    *xi = 2.0 * R.t4[a] - 1.0;
    *eta = 2.0 * R.t4[b] - 1.0;
    *w = 4.0 * R.w4[a] * R.w4[b];
  } else if (cls == 1) {
    const int a = p / 8, b = p % 8;
    *xi = 2.0 * R.t8[a] - 1.0;
    *eta = 2.0 * R.t8[b] - 1.0;
    *w = 4.0 * R.w8[a] * R.w8[b];
  } else {
    // quarters [-1,0]x[-1,0], [0,1]x[-1,0], [-1,0]x[0,1], [0,1]x[0,1]
    const int qd = p / 64, a = (p % 64) / 8, b = p % 8;
    *xi = ((qd & 1) ? 0.0 : -1.0) + R.t8[a];
    *eta = ((qd & 2) ? 0.0 : -1.0) + R.t8[b];
    *w = R.w8[a] * R.w8[b];
  }
}

// Quadrature point of a class rule: y, unit normal, weight w |J| (7 values).
__host__ __device__ inline void q9_table_point(const double a[9][3], const Q9Rules& R, int cls, int p,
                                               double out[7]) {
  double xi, eta, w, y[3], yx[3], ye[3], J[3];
  q9_rule_point(R, cls, p, &xi, &eta, &w);
  q9_eval(a, xi, eta, y, yx, ye);
  q9_cross(yx, ye, J);
  const double dJ = sqrt(q9_dot(J, J));
  for (int d = 0; d < 3; ++d) {
    out[d] = y[d];
    out[3 + d] = J[d] / dJ;
  }
  out[6] = w * dJ;
}

// Centre, normal, chord and area of an element; false if its Jacobian
// vanishes (relative to the chord) at the centre or at a far-rule point.
__host__ __device__ inline bool q9_prepare(const double Y[9][3], const Q9Rules& R, Q9Elem& E) {
  double a[9][3];
  q9_monomials(Y, a);
  for (int n = 0; n < 9; ++n)
    for (int d = 0; d < 3; ++d) E.Y[n][d] = Y[n][d];
  const int corner[4] = {0, 2, 8, 6};
  double h = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double* u = Y[corner[c]];
    const double* v = Y[corner[(c + 1) % 4]];
    const double dv[3] = {v[0] - u[0], v[1] - u[1], v[2] - u[2]};
    h = fmax(h, sqrt(q9_dot(dv, dv)));
  }
  E.hmax = h;
  double J[3];
  q9_cross(a[1], a[3], J);
  const double J0 = sqrt(q9_dot(J, J));
  for (int d = 0; d < 3; ++d) {
    E.c[d] = a[0][d];
    E.nrm[d] = J0 > 0.0 ? J[d] / J0 : 0.0;
  }
  bool ok = J0 > 1e-12 * h * h;
  double area = 0.0;
  for (int p = 0; p < Q9_FAR; ++p) {
    double t[7];
    q9_table_point(a, R, 0, p, t);
    area += t[6];
    double xi, eta, w;
    q9_rule_point(R, 0, p, &xi, &eta, &w);
    ok = ok && t[6] > 1e-12 * h * h * w;
  }
  E.area = area;
  return ok && h > 0.0;
}

// The four Burton-Miller integrands at one point, weight w, d = x - y:
// D += w dG/dn_y, H += w d2G/dn_x dn_y and with SK also S += w G,
// K += w dG/dn_x (G = e^{ikr}/(4 pi r), the normals of the mesh).
template <bool SK>
__host__ __device__ inline void q9_kernels(const double dv[3], const double nx[3], const double ny[3], double w,
                                           double k, cd& D, cd& H, cd& S, cd& K) {
  const double r2 = q9_dot(dv, dv);
  const double r = sqrt(r2);
  const double ir = 1.0 / r;
  const double kr = k * r;
  double s, c;
  sincos(kr, &s, &c);
  const double dny = q9_dot(dv, ny), dnx = q9_dot(dv, nx), nn = q9_dot(nx, ny);
  const double inv4pi = 0.25 / PI;
  const double ir3 = ir * ir * ir;
  // a = e^{ikr}(1 - ikr), b = e^{ikr}(3 - k^2 r^2 - 3ikr)
  const double a_re = c + s * kr, a_im = s - c * kr;
  const double f = w * dny * ir3 * inv4pi;
  D.x += a_re * f;
  D.y += a_im * f;
  const double t = 3.0 - kr * kr;
  const double b_re = c * t + 3.0 * s * kr, b_im = s * t - 3.0 * c * kr;
  const double g1 = w * nn * ir3 * inv4pi;
  const double g2 = w * dnx * dny * ir3 * ir * ir * inv4pi;
  H.x += a_re * g1 - b_re * g2;
  H.y += a_im * g1 - b_im * g2;
  if (SK) {
    const double gs = w * ir * inv4pi;
    S.x += c * gs;
    S.y += s * gs;
    const double gk = -w * dnx * ir3 * inv4pi;
    K.x += a_re * gk;
    K.y += a_im * gk;
  }
}

// Sum over points p0, p0 + stride, ... < npts of a table of 8-double points
// (y, n_y, w|J|, pad), the element translated by shift, seen from (x, nx).
template <bool SK>
__host__ __device__ inline void q9_sum_table(const double* tab, int npts, int p0, int stride, const double x[3],
                                             const double nx[3], const double sh[3], double k, cd& D, cd& H, cd& S,
                                             cd& K) {
  for (int p = p0; p < npts; p += stride) {
    const double* q = tab + 8 * (size_t)p;
    const double dv[3] = {x[0] - (q[0] + sh[0]), x[1] - (q[1] + sh[1]), x[2] - (q[2] + sh[2])};
    const double ny[3] = {q[3], q[4], q[5]};
    q9_kernels<SK>(dv, nx, ny, q[6], k, D, H, S, K);
  }
}

// Element centre quantities of the self rule.
struct Q9Centre {
  double a[9][3];   // monomial coefficients
  double J0;        // |y_xi x y_eta| at the centre
  double nx[3];     // unit normal at the centre
  double Jv[3];     // y_xi x y_eta at the centre
  double Jx[3];     // d/dxi of y_xi x y_eta at the centre
  double Je[3];     // d/deta of y_xi x y_eta at the centre
};
__host__ __device__ inline void q9_centre(const double Y[9][3], Q9Centre& C) {
  q9_monomials(Y, C.a);
  const double* a10 = C.a[1];
  const double* a01 = C.a[3];
  const double* a11 = C.a[4];
  double a20x2[3], a02x2[3];
  for (int d = 0; d < 3; ++d) {
    a20x2[d] = 2.0 * C.a[2][d];
    a02x2[d] = 2.0 * C.a[6][d];
  }
  q9_cross(a10, a01, C.Jv);
  C.J0 = sqrt(q9_dot(C.Jv, C.Jv));
  for (int d = 0; d < 3; ++d) C.nx[d] = C.Jv[d] / C.J0;
  double u[3], v[3];
  q9_cross(a20x2, a01, u);   // y_xixi x y_eta
  q9_cross(a10, a11, v);     // y_xi x y_xieta
  for (int d = 0; d < 3; ++d) C.Jx[d] = u[d] + v[d];
  q9_cross(a11, a01, u);     // y_xieta x y_eta
  q9_cross(a10, a02x2, v);   // y_xi x y_etaeta
  for (int d = 0; d < 3; ++d) C.Je[d] = u[d] + v[d];
}

// Contribution of angular node it (0 .. Q9_THETA-1) of the self rule to
// D, H (finite part), S, K of the element at its own centre.
template <bool SK>
__host__ __device__ inline void q9_self_theta(const Q9Centre& C, const Q9Rules& R, double k, int it, cd& D, cd& H,
                                              cd& S, cd& K) {
  const int side = it / 16, m = it % 16;
  const double half_pi = 0.5 * PI;
  const double th = -0.25 * PI + side * half_pi + half_pi * R.t16[m];
  const double wth = half_pi * R.w16[m];
  double sn, cs;
  sincos(th, &sn, &cs);
  const double rhat = side == 0 ? 1.0 / cs : side == 1 ? 1.0 / sn : side == 2 ? -1.0 / cs : -1.0 / sn;
  const double (*a)[3] = C.a;
  // y - x = rho (A + rho (B + rho (C3 + rho C4)))
  double A[3], B[3], C3[3], C4[3];
  for (int d = 0; d < 3; ++d) {
    A[d] = a[1][d] * cs + a[3][d] * sn;
    B[d] = a[2][d] * cs * cs + a[4][d] * cs * sn + a[6][d] * sn * sn;
    C3[d] = a[5][d] * cs * cs * sn + a[7][d] * cs * sn * sn;
    C4[d] = a[8][d] * cs * cs * sn * sn;
  }
  const double beta = sqrt(q9_dot(A, A));
  const double AB = q9_dot(A, B);
  const double J1 = (C.Jv[0] * (C.Jx[0] * cs + C.Je[0] * sn) + C.Jv[1] * (C.Jx[1] * cs + C.Je[1] * sn) +
                     C.Jv[2] * (C.Jx[2] * cs + C.Je[2] * sn)) / C.J0;
  const double inv4pi = 0.25 / PI;
  const double b3 = beta * beta * beta;
  const double Fm2 = C.J0 * inv4pi / b3;
  const double Fm1 = (J1 - 3.0 * C.J0 * AB / (beta * beta)) * inv4pi / b3;
  cd Dt = mkc(0.0, 0.0), St = mkc(0.0, 0.0), Kt = mkc(0.0, 0.0), inner = mkc(0.0, 0.0);
  for (int s = 0; s < Q9_RHO; ++s) {
    const double rho = rhat * R.t16[s];
    const double wu = R.w16[s] * rhat;
    double dv[3];
    for (int d = 0; d < 3; ++d) dv[d] = -rho * (A[d] + rho * (B[d] + rho * (C3[d] + rho * C4[d])));
    double y[3], yx[3], ye[3], J[3];
    q9_eval(a, rho * cs, rho * sn, y, yx, ye);
    q9_cross(yx, ye, J);
    const double dJ = sqrt(q9_dot(J, J));
    const double ny[3] = {J[0] / dJ, J[1] / dJ, J[2] / dJ};
    cd Dp = mkc(0.0, 0.0), Hp = mkc(0.0, 0.0), Sp = mkc(0.0, 0.0), Kp = mkc(0.0, 0.0);
    q9_kernels<SK>(dv, C.nx, ny, rho * dJ, k, Dp, Hp, Sp, Kp);   // integrands x |J| rho
    Dt = cadd(Dt, cmulr(Dp, wu));
    inner = cadd(inner, cmulr(mkc(Hp.x - Fm2 / (rho * rho) - Fm1 / rho, Hp.y), wu));
    if (SK) {
      St = cadd(St, cmulr(Sp, wu));
      Kt = cadd(Kt, cmulr(Kp, wu));
    }
  }
  D = cadd(D, cmulr(Dt, wth));
  const double extra = Fm1 * log(rhat * beta) + Fm2 * (AB / (beta * beta) - 1.0 / rhat);
  H = cadd(H, cmulr(mkc(inner.x + extra, inner.y), wth));
  if (SK) {
    S = cadd(S, cmulr(St, wth));
    K = cadd(K, cmulr(Kt, wth));
  }
}

}  // namespace fmpb

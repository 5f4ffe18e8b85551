// Discontinuous pressure of order 1 or 2 on the nine-node quadrilaterals
// (the paper's variable-order pressure, Sec. 2.1 and Eq. (matrixBEM)):
// shape functions, collocation nodes, the order-dependent very-near rule and
// the singular self rule about an off-centre node.  Host-and-device code,
// used by the kernels of quad9p.cu.
//
//   order 1: 2 x 2 nodes at (+-s1, +-s1), s1 = 1/sqrt(3), bilinear Lagrange,
//            node (i, j) at 2 j + i;
//   order 2: the eight-node serendipity element on [-s2, s2]^2,
//            s2 = sqrt(3/5), nodes counter-clockwise from (-s2, -s2):
//            (-,-) (0,-) (+,-) (+,0) (+,+) (0,+) (-,+) (-,0).
// Rules: very near (d < 1.5 h) 8 x 8 Gauss-Legendre on each of 4 x 4
// (order 1) or 8 x 8 (order 2) parameter sub-squares; self: polar
// coordinates about the node (the square cut into four triangles with apex
// there), 24 Gauss-Legendre nodes in theta per triangle and 24 in rho.
// The self rule forms y - x from the monomial coefficients of the map about
// the node (b_pq of y(xi_a + u, eta_a + v) = sum b_pq u^p v^q), and the
// finite part of N_b H uses G_-2 = F_-2 N_b0, G_-1 = F_-1 N_b0 + F_-2 N_b1,
// N_b1 = grad N_b . (cos, sin), with the (A.B) and log terms kept.
#pragma once
#include "quad9.cuh"

namespace fmpb {

constexpr int Q9P_MAXNB = 8;
constexpr int Q9P_Q = 24;               // self rule: nodes per direction
constexpr int Q9P_THETA = 4 * Q9P_Q;    // angular nodes of the self rule

// Order 0 (one constant per element at the centre, N = 1) is included for
// the kernels that serve every order (image blocks, field points).
struct Q9Basis {
  int order;   // 0, 1 or 2
  int nb;      // 1, 4 or 8
  double s;    // node half-width: 0, 1/sqrt(3) or sqrt(3/5)
};

__host__ __device__ inline Q9Basis q9p_basis(int order) {
  Q9Basis b;
  b.order = order;
  b.nb = order == 0 ? 1 : order == 1 ? 4 : 8;
  b.s = order == 0 ? 0.0 : order == 1 ? 1.0 / sqrt(3.0) : sqrt(3.0 / 5.0);
  return b;
}

// Parameter coordinates of node a.
__host__ __device__ inline void q9p_node(const Q9Basis& B, int a, double* xi, double* eta) {
  if (B.order == 0) {
    *xi = 0.0;
    *eta = 0.0;
    return;
  }
  if (B.order == 1) {
    *xi = (a & 1) ? B.s : -B.s;
    *eta = (a & 2) ? B.s : -B.s;
    return;
  }
  const int u[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
  const int v[8] = {-1, -1, -1, 0, 1, 1, 1, 0};
  *xi = B.s * u[a];
  *eta = B.s * v[a];
}

// N_b and, if G is not null, dN_b/dxi, dN_b/deta at (xi, eta).
__host__ __device__ inline void q9p_shape(const Q9Basis& B, double xi, double eta, double N[Q9P_MAXNB],
                                          double G[Q9P_MAXNB][2]) {
  if (B.order == 0) {
    N[0] = 1.0;
    if (G) G[0][0] = G[0][1] = 0.0;
    return;
  }
  if (B.order == 1) {
    const double h = 0.5 / B.s;
    const double l[2] = {(B.s - xi) * h, (B.s + xi) * h};
    const double m[2] = {(B.s - eta) * h, (B.s + eta) * h};
    const double dl[2] = {-h, h};
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i) {
        N[2 * j + i] = l[i] * m[j];
        if (G) {
          G[2 * j + i][0] = dl[i] * m[j];
          G[2 * j + i][1] = l[i] * dl[j];
        }
      }
    return;
  }
  const double is = 1.0 / B.s;
  const double u = xi * is, v = eta * is;
  const int ua[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
  const int va[8] = {-1, -1, -1, 0, 1, 1, 1, 0};
  for (int a = 0; a < 8; ++a) {
    const double uu = ua[a], vv = va[a];
    double n, du, dv;
    if (ua[a] != 0 && va[a] != 0) {
      n = 0.25 * (1 + u * uu) * (1 + v * vv) * (u * uu + v * vv - 1);
      du = 0.25 * uu * (1 + v * vv) * (2 * u * uu + v * vv);
      dv = 0.25 * vv * (1 + u * uu) * (u * uu + 2 * v * vv);
    } else if (ua[a] == 0) {
      n = 0.5 * (1 - u * u) * (1 + v * vv);
      du = -u * (1 + v * vv);
      dv = 0.5 * vv * (1 - u * u);
    } else {
      n = 0.5 * (1 + u * uu) * (1 - v * v);
      du = 0.5 * uu * (1 - v * v);
      dv = -v * (1 + u * uu);
    }
    N[a] = n;
    if (G) {
      G[a][0] = du * is;
      G[a][1] = dv * is;
    }
  }
}

// Parameter point and weight of point p of the very-near rule of an order:
// parts x parts sub-squares (parts = 2, 4 or 8; 2 is the quarter rule of
// order 0, in the same order), 8 x 8 Gauss-Legendre each,
// sub-square (i, j) at p / 64 = j parts + i, point (a, b) at p % 64 = 8 a + b.
__host__ __device__ inline void q9p_vnear_point(const Q9Rules& R, int parts, int p, double* xi, double* eta,
                                                double* w) {
  const int sq = p / 64, i = sq % parts, j = sq / parts;
  const int a = (p % 64) / 8, b = p % 8;
  const double hs = 2.0 / parts;
  *xi = -1.0 + hs * (i + R.t8[a]);
  *eta = -1.0 + hs * (j + R.t8[b]);
  *w = hs * hs * R.w8[a] * R.w8[b];
}

// Near (8 x 8 on the element) or very-near (order-dependent sub-squares)
// regular integrals of element Y translated by sh, seen from (x, nx), for
// every shape N_b: points p0, p0 + stride, ... of the rule.
template <bool SK>
__host__ __device__ inline void q9p_near_sum(const double Y[9][3], const Q9Basis& B, const Q9Rules& R, bool very,
                                             const double x[3], const double nx[3], const double sh[3], double k,
                                             int p0, int stride, cd* D, cd* H, cd* S, cd* K) {
  double am[9][3];
  q9_monomials(Y, am);
  const int parts = B.order == 0 ? 2 : B.order == 1 ? 4 : 8;
  const int npts = very ? 64 * parts * parts : 64;
  for (int p = p0; p < npts; p += stride) {
    double xi, eta, w;
    if (very)
      q9p_vnear_point(R, parts, p, &xi, &eta, &w);
    else
      q9_rule_point(R, 1, p, &xi, &eta, &w);
    double y[3], yx[3], ye[3], J[3];
    q9_eval(am, xi, eta, y, yx, ye);
    q9_cross(yx, ye, J);
    const double dJ = sqrt(q9_dot(J, J));
    const double ny[3] = {J[0] / dJ, J[1] / dJ, J[2] / dJ};
    const double dv[3] = {x[0] - (y[0] + sh[0]), x[1] - (y[1] + sh[1]), x[2] - (y[2] + sh[2])};
    cd Dp = mkc(0.0, 0.0), Hp = mkc(0.0, 0.0), Sp = mkc(0.0, 0.0), Kp = mkc(0.0, 0.0);
    q9_kernels<SK>(dv, nx, ny, w * dJ, k, Dp, Hp, Sp, Kp);
    double N[Q9P_MAXNB];
    q9p_shape(B, xi, eta, N, nullptr);
    for (int c = 0; c < B.nb; ++c) {
      D[c] = cadd(D[c], cmulr(Dp, N[c]));
      H[c] = cadd(H[c], cmulr(Hp, N[c]));
      if (SK) {
        S[c] = cadd(S[c], cmulr(Sp, N[c]));
        K[c] = cadd(K[c], cmulr(Kp, N[c]));
      }
    }
  }
}

// Contribution of one element (nodes Y, centre cen, chord hmax; translated
// by sh) to the pressure at a field point x: int (dG/dn_y + i k beta G) p dA
// with p = sum_b N_b pd[b] (order 0: p = pd[0]), by the class rules of the
// collocation points (order 0: quarters for the very-near class; orders 1, 2:
// their sub-squares).  ikb = i k beta; SK: with the single layer; dsign = -1
// for a mirrored element whose nodes kept their order (computed normal -R n).
template <bool SK>
__host__ __device__ inline cd q9_field_element(const double Y[9][3], const double cen[3], double hmax, int order,
                                               const Q9Rules& R, const double x[3], const double sh[3], double k,
                                               cd ikb, double dsign, const cd* pd) {
  double dc[3];
  for (int d = 0; d < 3; ++d) dc[d] = x[d] - (cen[d] + sh[d]);
  const double dist = sqrt(q9_dot(dc, dc));
  const int cls = dist >= FAR_RATIO * hmax ? 0 : dist >= NEAR_RATIO * hmax ? 1 : 2;
  const int parts = order == 0 ? 2 : order == 1 ? 4 : 8;
  const int npts = cls == 0 ? Q9_FAR : cls == 1 ? Q9_NEAR : 64 * parts * parts;
  const Q9Basis B = q9p_basis(order == 0 ? 1 : order);
  double am[9][3];
  q9_monomials(Y, am);
  const double nz[3] = {0.0, 0.0, 1.0};   // the integrands used here do not read n_x
  cd acc = mkc(0.0, 0.0);
  for (int p = 0; p < npts; ++p) {
    double xi, eta, w;
    if (cls == 2 && order > 0)
      q9p_vnear_point(R, parts, p, &xi, &eta, &w);
    else
      q9_rule_point(R, cls, p, &xi, &eta, &w);
    double y[3], yx[3], ye[3], J[3];
    q9_eval(am, xi, eta, y, yx, ye);
    q9_cross(yx, ye, J);
    const double dJ = sqrt(q9_dot(J, J));
    const double ny[3] = {J[0] / dJ, J[1] / dJ, J[2] / dJ};
    const double dv[3] = {x[0] - (y[0] + sh[0]), x[1] - (y[1] + sh[1]), x[2] - (y[2] + sh[2])};
    cd Dp = mkc(0.0, 0.0), Hp = mkc(0.0, 0.0), Sp = mkc(0.0, 0.0), Kp = mkc(0.0, 0.0);
    q9_kernels<SK>(dv, nz, ny, w * dJ, k, Dp, Hp, Sp, Kp);
    cd dens = pd[0];
    if (order > 0) {
      double N[Q9P_MAXNB];
      q9p_shape(B, xi, eta, N, nullptr);
      dens = mkc(0.0, 0.0);
      for (int b = 0; b < B.nb; ++b) dens = cadd(dens, cmulr(pd[b], N[b]));
    }
    Dp = cmulr(Dp, dsign);
    const cd g = SK ? cfma(ikb, Sp, Dp) : Dp;
    acc = cfma(g, dens, acc);
  }
  return acc;
}

// Monomial coefficients of the map about (xa, ea): y(xa + u, ea + v) =
// sum_{p,q} b[3 q + p] u^p v^q, from those about the centre.
__host__ __device__ inline void q9p_shift_monomials(const double a[9][3], double xa, double ea, double b[9][3]) {
  const double xp[3] = {1.0, xa, xa * xa}, ep[3] = {1.0, ea, ea * ea};
  const double binom[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};   // C(P, p)
  for (int q = 0; q < 3; ++q)
    for (int p = 0; p < 3; ++p)
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int Q = q; Q < 3; ++Q)
          for (int P = p; P < 3; ++P)
            s += a[3 * Q + P][d] * binom[P][p] * binom[Q][q] * xp[P - p] * ep[Q - q];
        b[3 * q + p][d] = s;
      }
}

// Quantities of the self rule about node a of one element.
struct Q9Node {
  double b[9][3];   // monomials about the node
  double xa, ea;    // the node in the parameter square
  double J0;
  double nx[3];
  double Jv[3], Jx[3], Je[3];
  double N0[Q9P_MAXNB];       // N_b at the node
  double G0[Q9P_MAXNB][2];    // grad N_b at the node
  double ang[5];              // corner angles (increasing) of the four triangles
};

__host__ __device__ inline void q9p_node_setup(const double Y[9][3], const Q9Basis& B, int a, Q9Node& Nd) {
  double am[9][3];
  q9_monomials(Y, am);
  q9p_node(B, a, &Nd.xa, &Nd.ea);
  q9p_shift_monomials(am, Nd.xa, Nd.ea, Nd.b);
  const double* b10 = Nd.b[1];
  const double* b01 = Nd.b[3];
  const double* b11 = Nd.b[4];
  double b20x2[3], b02x2[3];
  for (int d = 0; d < 3; ++d) {
    b20x2[d] = 2.0 * Nd.b[2][d];
    b02x2[d] = 2.0 * Nd.b[6][d];
  }
  q9_cross(b10, b01, Nd.Jv);
  Nd.J0 = sqrt(q9_dot(Nd.Jv, Nd.Jv));
  for (int d = 0; d < 3; ++d) Nd.nx[d] = Nd.Jv[d] / Nd.J0;
  double u[3], v[3];
  q9_cross(b20x2, b01, u);
  q9_cross(b10, b11, v);
  for (int d = 0; d < 3; ++d) Nd.Jx[d] = u[d] + v[d];
  q9_cross(b11, b01, u);
  q9_cross(b10, b02x2, v);
  for (int d = 0; d < 3; ++d) Nd.Je[d] = u[d] + v[d];
  q9p_shape(B, Nd.xa, Nd.ea, Nd.N0, Nd.G0);
  const double cx[4] = {1.0, 1.0, -1.0, -1.0}, cy[4] = {-1.0, 1.0, 1.0, -1.0};
  for (int c = 0; c < 4; ++c) Nd.ang[c] = atan2(cy[c] - Nd.ea, cx[c] - Nd.xa);
  for (int c = 1; c < 4; ++c)
    while (Nd.ang[c] <= Nd.ang[c - 1]) Nd.ang[c] += 2.0 * PI;
  Nd.ang[4] = Nd.ang[0] + 2.0 * PI;
}

// Contribution of angular node it (0 .. Q9P_THETA-1) of the self rule about
// the node to D, H (finite part), S, K of every shape N_b of the element.
// t24, w24: Gauss-Legendre of order 24 on [0, 1].
template <bool SK>
__host__ __device__ inline void q9p_self_theta(const Q9Node& Nd, const Q9Basis& B, const double* t24,
                                               const double* w24, double k, int it, cd* D, cd* H, cd* S,
                                               cd* K) {
  const int side = it / Q9P_Q, m = it % Q9P_Q;
  const double t0 = Nd.ang[side], t1 = Nd.ang[side + 1];
  const double th = t0 + (t1 - t0) * t24[m];
  const double wth = (t1 - t0) * w24[m];
  double sn, cs;
  sincos(th, &sn, &cs);
  const double rhat = side == 0 ? (1.0 - Nd.xa) / cs
                    : side == 1 ? (1.0 - Nd.ea) / sn
                    : side == 2 ? (-1.0 - Nd.xa) / cs
                                : (-1.0 - Nd.ea) / sn;
  const double (*b)[3] = Nd.b;
  // y - x = rho (A + rho (Bq + rho (C3 + rho C4)))
  double A[3], Bq[3], C3[3], C4[3];
  for (int d = 0; d < 3; ++d) {
    A[d] = b[1][d] * cs + b[3][d] * sn;
    Bq[d] = b[2][d] * cs * cs + b[4][d] * cs * sn + b[6][d] * sn * sn;
    C3[d] = b[5][d] * cs * cs * sn + b[7][d] * cs * sn * sn;
    C4[d] = b[8][d] * cs * cs * sn * sn;
  }
  const double beta = sqrt(q9_dot(A, A));
  const double AB = q9_dot(A, Bq);
  const double J1 = (Nd.Jv[0] * (Nd.Jx[0] * cs + Nd.Je[0] * sn) + Nd.Jv[1] * (Nd.Jx[1] * cs + Nd.Je[1] * sn) +
                     Nd.Jv[2] * (Nd.Jx[2] * cs + Nd.Je[2] * sn)) / Nd.J0;
  const double inv4pi = 0.25 / PI;
  const double b3 = beta * beta * beta;
  const double Fm2 = Nd.J0 * inv4pi / b3;
  const double Fm1 = (J1 - 3.0 * Nd.J0 * AB / (beta * beta)) * inv4pi / b3;
  const int nb = B.nb;
  // the (A.B) and log terms of the finite part
  const double lnrb = log(rhat * beta), corr = AB / (beta * beta) - 1.0 / rhat;
  for (int c = 0; c < nb; ++c) {
    const double g2 = Fm2 * Nd.N0[c];
    const double g1 = Fm1 * Nd.N0[c] + Fm2 * (Nd.G0[c][0] * cs + Nd.G0[c][1] * sn);
    H[c].x += wth * (g1 * lnrb + g2 * corr);
  }
  for (int s = 0; s < Q9P_Q; ++s) {
    const double rho = rhat * t24[s];
    const double wq = wth * w24[s] * rhat;
    double dv[3];
    for (int d = 0; d < 3; ++d) dv[d] = -rho * (A[d] + rho * (Bq[d] + rho * (C3[d] + rho * C4[d])));
    double y[3], yx[3], ye[3], J[3];
    q9_eval(b, rho * cs, rho * sn, y, yx, ye);
    q9_cross(yx, ye, J);
    const double dJ = sqrt(q9_dot(J, J));
    const double ny[3] = {J[0] / dJ, J[1] / dJ, J[2] / dJ};
    cd Dp = mkc(0.0, 0.0), Hp = mkc(0.0, 0.0), Sp = mkc(0.0, 0.0), Kp = mkc(0.0, 0.0);
    q9_kernels<SK>(dv, Nd.nx, ny, rho * dJ, k, Dp, Hp, Sp, Kp);   // integrands x |J| rho
    double N[Q9P_MAXNB];
    q9p_shape(B, Nd.xa + rho * cs, Nd.ea + rho * sn, N, nullptr);
    const double ir = 1.0 / rho;
    for (int c = 0; c < nb; ++c) {
      const double f = wq * N[c];
      const double g2 = Fm2 * Nd.N0[c];
      const double g1 = Fm1 * Nd.N0[c] + Fm2 * (Nd.G0[c][0] * cs + Nd.G0[c][1] * sn);
      D[c] = cadd(D[c], cmulr(Dp, f));
      H[c].x += wq * (Hp.x * N[c] - (g2 * ir + g1) * ir);
      H[c].y += f * Hp.y;
      if (SK) {
        S[c] = cadd(S[c], cmulr(Sp, f));
        K[c] = cadd(K[c], cmulr(Kp, f));
      }
    }
  }
}

}  // namespace fmpb

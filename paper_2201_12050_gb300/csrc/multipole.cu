// Single-level FMM operators of the FMPBEM (Sec. 3.1-3.2, Appendix A):
// P2M table V_0 (Eq. (p2m)), L2P table U_0 (Eq. (l2p) and its normal
// derivative), M2L blocks K(delta) (Eqs. (m2l), (wigner)) and the P2M / L2P
// applications of the matrix-vector product (Sec. 3.5).
//
// Conventions (readings of points the paper leaves open or prints garbled):
//   Y_n^m = s_m sqrt((n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{i m phi},
//     Ferrers P without the Condon-Shortley phase, s_m = (-1)^m for m < 0
//     (negative orders by Rodrigues' formula);
//   I_n^m(x) = j_n(k|x|) Y_n^m, O_n^m(x) = h_n^(1)(k|x|) Y_n^m (k restored);
//   W = (2l+1) i^{n-n'+l} (n n' l; 0 0 0)(n n' l; m m' -m-m'), l from
//     max(|m+m'|, |n-n'|) to n+n' with n+n'-l even;
//   coefficient (n, m) at q = n(n+1) + m, B = (n_t+1)^2.
// With mesh normals n_m (into the fluid) the far part of the collocation
// operator is U_0 K V_0 with
//   V_0[q][j] = int_{E_j} conj(n_m . grad I_q)(y - y_c) dA        (far rule),
//   U_0[i][q] = -(ik/4pi)(2n+1)[conj(I_q) + (i/k) conj(n_m . grad I_q)](x_i - x_c),
//   K(d)[q][q'] = (2n'+1)(-1)^{m+m'} sum_l W O_l^{m+m'}(d),  d = x_c - y_c.
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "multipole.cuh"
#include "ff.cuh"
#include "quad9p.cuh"

namespace fmpb {

// -------------------------------------------------- double-double (Dekker) --
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_make(double a) { return {a, 0.0}; }
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  double e = s.lo + x.lo + y.lo;
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  double p = __dmul_rn(x.hi, y.hi);
  double e = fma(x.hi, y.hi, -p);
  e += x.hi * y.lo + x.lo * y.hi;
  return quick_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul_d(dd x, double y) {
  double p = __dmul_rn(x.hi, y);
  double e = fma(x.hi, y, -p);
  e += x.lo * y;
  return quick_two_sum(p, e);
}
__device__ dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_add(x, dd_neg(dd_mul_d(y, q1)));
  double q2 = r.hi / y.hi;
  r = dd_add(r, dd_neg(dd_mul_d(y, q2)));
  double q3 = r.hi / y.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd_make(q3));
}
__device__ dd dd_sqrt(dd x) {
  if (x.hi <= 0.0) return dd_make(0.0);
  double s = sqrt(x.hi);
  // one Newton step: s + (x - s^2) / (2 s)
  dd s2 = dd_mul(dd_make(s), dd_make(s));
  dd r = dd_add(x, dd_neg(s2));
  return dd_add(dd_make(s), dd_make(r.hi / (2.0 * s)));
}

// Wigner 3j symbol by Racah's single-sum formula, every factorial, product
// and the alternating sum in double-double (about 32 digits), rounded once.
__device__ double wigner3j_dd(int j1, int j2, int j3, int m1, int m2, int m3, const dd* fact) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
  dd tri = dd_div(dd_mul(dd_mul(fact[j1 + j2 - j3], fact[j1 - j2 + j3]), fact[-j1 + j2 + j3]), fact[j1 + j2 + j3 + 1]);
  dd pref = dd_mul(tri, dd_mul(dd_mul(fact[j1 + m1], fact[j1 - m1]), dd_mul(fact[j2 + m2], fact[j2 - m2])));
  pref = dd_mul(pref, dd_mul(fact[j3 + m3], fact[j3 - m3]));
  int tmin = max(0, max(j2 - j3 - m1, j1 - j3 + m2));
  int tmax = min(j1 + j2 - j3, min(j1 - m1, j2 + m2));
  dd s = dd_make(0.0);
  for (int t = tmin; t <= tmax; ++t) {
    dd den = dd_mul(dd_mul(fact[t], fact[j3 - j2 + t + m1]), dd_mul(fact[j3 - j1 + t - m2], fact[j1 + j2 - j3 - t]));
    den = dd_mul(den, dd_mul(fact[j1 - t - m1], fact[j2 - t + m2]));
    dd term = dd_div(dd_make(1.0), den);
    s = dd_add(s, (t & 1) ? dd_neg(term) : term);
  }
  dd v = dd_mul(s, dd_sqrt(pref));
  double sign = ((j1 - j2 - m3) & 1) ? -1.0 : 1.0;
  return sign * (v.hi + v.lo);
}

// W3[((q*B + q') * (nt+1)) + (l - lmin)/2] = (2l+1)(n n' l;000)(n n' l; m m' -m-m'),
// lmin = max(|m+m'|, |n-n'|) rounded up to the parity of n+n'.
__global__ void k_wigner_table(int nt, double* __restrict__ W3) {
  __shared__ dd fact[4 * MAX_NT + 2];
  if (threadIdx.x == 0) {
    fact[0] = dd_make(1.0);
    for (int i = 1; i < 4 * nt + 2; ++i) fact[i] = dd_mul_d(fact[i - 1], (double)i);
  }
  __syncthreads();
  const int B = (nt + 1) * (nt + 1);
  const int L = nt + 1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * B * L;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int li = (int)(idx % L);
    const int qq = (int)(idx / L);
    const int q = qq / B, qp = qq % B;
    int n, m, n2, m2;
    q_to_nm(q, n, m);
    q_to_nm(qp, n2, m2);
    const int mu = m + m2;
    int lmin = max(abs(mu), abs(n - n2));
    if ((n + n2 - lmin) & 1) ++lmin;
    const int l = lmin + 2 * li;
    double v = 0.0;
    if (l <= n + n2) {
      double a = wigner3j_dd(n, n2, l, 0, 0, 0, fact);
      if (a != 0.0) v = (2 * l + 1) * a * wigner3j_dd(n, n2, l, m, m2, -mu, fact);
    }
    W3[idx] = v;
  }
}

// ------------------------------------------------------ special functions --
// Spherical Bessel j_0..j_nmax at x >= 0: power series below 0.5, Miller's
// backward recurrence normalised by sum_n (2n+1) j_n^2 = 1 above.
__device__ void sph_bessel_j(int nmax, double x, double* j) {
  if (x < 0.5) {
    double xn = 1.0, dfact = 1.0;   // x^n, (2n+1)!!
    for (int n = 0; n <= nmax; ++n) {
      if (n > 0) {
        xn *= x;
        dfact *= (2 * n + 1);
      }
      double term = 1.0, sum = 1.0, y = -0.5 * x * x;
      for (int k = 1; k < 30; ++k) {
        term *= y / (k * (2.0 * n + 2 * k + 1));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      j[n] = xn / dfact * sum;
    }
    return;
  }
  int N0 = nmax + 24 + (int)(1.5 * x);
  double fp1 = 0.0, f = 1.0, norm = 0.0;
  for (int n = N0; n >= 0; --n) {
    // f = f_n (unnormalised); store n <= nmax
    if (n <= nmax) j[n] = f;
    norm += (2 * n + 1) * f * f;
    double fm1 = (2 * n + 1) / x * f - fp1;
    fp1 = f;
    f = fm1;
    if (fabs(f) > 1e120) {   // rescale to stay in range
      f *= 1e-120;
      fp1 *= 1e-120;
      norm *= 1e-240;
      for (int i = n; i <= nmax; ++i) j[i] *= 1e-120;
    }
  }
  double s = 1.0 / sqrt(norm);
  // sign from j_0 = sin x / x (or j_1 when j_0 is small)
  double j0 = sin(x) / x;
  double j1 = sin(x) / (x * x) - cos(x) / x;
  if (fabs(j0) >= fabs(j1)) {
    if ((j[0] < 0) != (j0 < 0)) s = -s;
  } else {
    if ((j[1] < 0) != (j1 < 0)) s = -s;
  }
  for (int n = 0; n <= nmax; ++n) j[n] *= s;
}

// Spherical Neumann y_0..y_nmax (x > 0) by the upward recurrence.
__device__ void sph_bessel_y(int nmax, double x, double* y) {
  double s, c;
  sincos(x, &s, &c);
  y[0] = -c / x;
  if (nmax >= 1) y[1] = -c / (x * x) - s / x;
  for (int n = 1; n < nmax; ++n) y[n + 1] = (2 * n + 1) / x * y[n] - y[n - 1];
}

// Angles of v: cos(theta), sin(theta), e^{i phi} (phi := 0 on the axis).
__device__ __forceinline__ void angles(const double v[3], double& r, double& ct, double& st, double& cp, double& sp) {
  r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  ct = r > 0.0 ? v[2] / r : 1.0;
  ct = fmin(1.0, fmax(-1.0, ct));
  double rho = sqrt(v[0] * v[0] + v[1] * v[1]);
  if (rho > 0.0) {
    cp = v[0] / rho;
    sp = v[1] / rho;
  } else {
    cp = 1.0;
    sp = 0.0;
  }
  st = sqrt(fmax(0.0, 1.0 - ct * ct));
}

// P[n*(nmax+1)+m] (no Condon-Shortley phase) and Q = P / sin(theta) (m >= 1).
__device__ void ferrers_tables(int nmax, double ct, double st, double* P, double* Q) {
  const int W = nmax + 1;
  double pmm = 1.0, qmm = 1.0;
  for (int m = 0; m <= nmax; ++m) {
    if (m > 0) pmm *= (2 * m - 1) * st;
    if (m > 1) qmm *= (2 * m - 1) * st;
    P[m * W + m] = pmm;
    if (Q) Q[m * W + m] = m >= 1 ? qmm : 0.0;
    if (m + 1 <= nmax) {
      P[(m + 1) * W + m] = (2 * m + 1) * ct * pmm;
      if (Q) Q[(m + 1) * W + m] = m >= 1 ? (2 * m + 1) * ct * qmm : 0.0;
    }
    for (int n = m + 2; n <= nmax; ++n) {
      P[n * W + m] = ((2 * n - 1) * ct * P[(n - 1) * W + m] - (n + m - 1) * P[(n - 2) * W + m]) / (n - m);
      if (Q)
        Q[n * W + m] = m >= 1 ? ((2 * n - 1) * ct * Q[(n - 1) * W + m] - (n + m - 1) * Q[(n - 2) * W + m]) / (n - m)
                              : 0.0;
    }
  }
}

// s_m sqrt((n-|m|)!/(n+|m|)!)
__device__ __forceinline__ double ynorm(int n, int m) {
  int am = abs(m);
  double r = 1.0;
  for (int i = n - am + 1; i <= n + am; ++i) r /= i;
  double v = sqrt(r);
  return (m < 0 && (am & 1)) ? -v : v;
}

// e^{i m phi} from e^{i phi} by repeated multiplication (m may be negative).
__device__ __forceinline__ cd eimphi(int m, double cp, double sp) {
  cd e = mkc(1.0, 0.0);
  cd b = m >= 0 ? mkc(cp, sp) : mkc(cp, -sp);
  for (int i = 0; i < abs(m); ++i) e = cmul(e, b);
  return e;
}

// Per-point tables of the regular waves, filled by one thread into shared
// memory and read by the threads that evaluate individual coefficients.
struct WaveSetup {
  double ct, st, cp, sp;
  double jb[MAX_NT + 3];
  double P[(MAX_NT + 2) * (MAX_NT + 2)];
  double Q[(MAX_NT + 2) * (MAX_NT + 2)];
  double rh[3], th[3], ph[3];
};

__device__ void wave_setup(int nt, const double v[3], double k, WaveSetup* w) {
  double r;
  angles(v, r, w->ct, w->st, w->cp, w->sp);
  sph_bessel_j(nt + 1, k * r, w->jb);
  ferrers_tables(nt + 1, w->ct, w->st, w->P, w->Q);
  w->rh[0] = w->st * w->cp; w->rh[1] = w->st * w->sp; w->rh[2] = w->ct;
  w->th[0] = w->ct * w->cp; w->th[1] = w->ct * w->sp; w->th[2] = -w->st;
  w->ph[0] = -w->sp; w->ph[1] = w->cp; w->ph[2] = 0.0;
}

// Regular wave I_q(v) and nrm . grad I_q(v) for one q from the tables.
// grad(j_n(kr) Y) = k[j_n'(x) Y r_hat + (j_n(x)/x)(dY/dtheta theta_hat
// + (i m/sin theta) Y phi_hat)], x = kr, with j_n' = (n j_{n-1} -
// (n+1) j_{n+1})/(2n+1) and j_n/x = (j_{n-1} + j_{n+1})/(2n+1), both
// regular at x = 0, and dP_n^m/dtheta = n cos Q_n^m - (n+m) Q_{n-1}^m
// (m >= 1), -P_n^1 (m = 0), Q = P / sin(theta).
__device__ void wave_eval(int nt, const WaveSetup& w, int q, const double nrm[3], double k, cd* I, cd* dI) {
  int n, m;
  q_to_nm(q, n, m);
  const int W = nt + 2;
  const int am = abs(m);
  const double jn = w.jb[n];
  const double jm1 = n > 0 ? w.jb[n - 1] : 0.0;
  const double jp1 = w.jb[n + 1];
  const double jd = n > 0 ? (n * jm1 - (n + 1) * jp1) / (2 * n + 1) : -jp1;
  const double jox = n > 0 ? (jm1 + jp1) / (2 * n + 1) : 0.0;   // n = 0 has no angular part
  const double N = ynorm(n, m);
  const cd e = eimphi(m, w.cp, w.sp);
  const double Pv = w.P[n * W + am];
  if (I) *I = cmulr(e, jn * N * Pv);
  if (dI) {
    double dP, qterm;
    if (am == 0) {
      dP = n >= 1 ? -w.P[n * W + 1] : 0.0;
      qterm = 0.0;
    } else {
      const double qn1 = (n - 1 >= am) ? w.Q[(n - 1) * W + am] : 0.0;
      dP = n * w.ct * w.Q[n * W + am] - (n + am) * qn1;
      qterm = w.Q[n * W + am];
    }
    const double nr = nrm[0] * w.rh[0] + nrm[1] * w.rh[1] + nrm[2] * w.rh[2];
    const double nth = nrm[0] * w.th[0] + nrm[1] * w.th[1] + nrm[2] * w.th[2];
    const double nph = nrm[0] * w.ph[0] + nrm[1] * w.ph[1] + nrm[2] * w.ph[2];
    // nrm.grad = k N e [ jd Pv nr + jox (dP nth + i m qterm nph) ]
    const double re = jd * Pv * nr + jox * dP * nth;
    const double im = jox * m * qterm * nph;
    *dI = cmulr(cmul(e, mkc(re, im)), k * N);
  }
}

// ---------------------------------------------------------------- tables --
// V_0[q][j]: far rule (collapsed Gauss-Legendre 3x3, apex v0) on element j.
// One CTA per element, one thread per coefficient.
__global__ void k_p2m_table(const Elem* __restrict__ el, int n, int nt, double k, cd beta, QuadRules qr,
                            const double* __restrict__ centres, cd* __restrict__ V0) {
  __shared__ WaveSetup ws;
  const int j = blockIdx.x;
  const Elem& E = el[j];
  const int B = (nt + 1) * (nt + 1);
  const int q = threadIdx.x;
  cd acc = mkc(0.0, 0.0);
  const cd ikb = mkc(-k * beta.y, k * beta.x);   // i k beta
  const double two_area = 2.0 * E.area;
  for (int a = 0; a < Q_FAR; ++a) {
    const double s = qr.t3[a];
    for (int b = 0; b < Q_FAR; ++b) {
      __syncthreads();
      if (threadIdx.x == 0) {
        double y[3];
        for (int d = 0; d < 3; ++d)
          y[d] = E.v[0][d] + s * ((E.v[1][d] - E.v[0][d]) + qr.t3[b] * (E.v[2][d] - E.v[1][d])) -
                 (centres ? centres[3 * j + d] : 0.0);
        wave_setup(nt, y, k, &ws);
      }
      __syncthreads();
      if (q < B) {
        cd I, dI;
        wave_eval(nt, ws, q, E.nrm, k, &I, &dI);
        const double w = two_area * s * qr.w3[a] * qr.w3[b];
        // conj(dI/dn) (double layer) + i k beta conj(I) (admittance single layer)
        const cd src = cadd(cconj(dI), cmul(ikb, cconj(I)));
        acc = cadd(acc, cmulr(src, w));
      }
    }
  }
  if (q < B) V0[(size_t)q * n + j] = acc;
}

// V_0[q][j] of a nine-node quadrilateral mesh: the far-class rule (4 x 4
// points, each with its own normal and weight w|J|) from the point-major
// table far_tab[(p 7 + f) n + j] (f: y, n_y, w|J|).  One CTA per element.
// dsign = -1 for the mirrored cell of a half-space operator (nodes kept in
// their order: computed normal -R n, the double-layer term changes sign).
__global__ void k_p2m_table_q9(const double* __restrict__ far_tab, int n, int nt, double k, cd beta,
                               double dsign, const double* __restrict__ centres, cd* __restrict__ V0) {
  __shared__ WaveSetup ws;
  const int j = blockIdx.x;
  const int B = (nt + 1) * (nt + 1);
  const int q = threadIdx.x;
  const size_t sn = (size_t)n;
  cd acc = mkc(0.0, 0.0);
  const cd ikb = mkc(-k * beta.y, k * beta.x);   // i k beta
  for (int p = 0; p < Q9_FAR; ++p) {
    const double* t = far_tab + (size_t)p * 7 * sn + j;
    __syncthreads();
    if (threadIdx.x == 0) {
      // about the cell origin, or about the element's own expansion centre
      const double y[3] = {t[0] - (centres ? centres[3 * j] : 0.0), t[sn] - (centres ? centres[3 * j + 1] : 0.0),
                           t[2 * sn] - (centres ? centres[3 * j + 2] : 0.0)};
      wave_setup(nt, y, k, &ws);
    }
    __syncthreads();
    if (q < B) {
      const double ny[3] = {t[3 * sn], t[4 * sn], t[5 * sn]};
      cd I, dI;
      wave_eval(nt, ws, q, ny, k, &I, &dI);
      const cd src = cadd(cmulr(cconj(dI), dsign), cmul(ikb, cconj(I)));
      acc = cadd(acc, cmulr(src, t[6 * sn]));
    }
  }
  if (q < B) V0[(size_t)q * n + j] = acc;
}

// V_0[q][f nb + b] with discontinuous pressure of order 1 or 2: the far rule
// of element f weighted by each shape N_b.  One CTA per element.
__global__ void k_p2m_table_q9p(const double* __restrict__ far_tab, int ne, int order, int nt, double k, cd beta,
                                Q9Rules R, double dsign, cd* __restrict__ V0) {
  __shared__ WaveSetup ws;
  const Q9Basis Bs = q9p_basis(order);
  const int f = blockIdx.x;
  const int B = (nt + 1) * (nt + 1);
  const int q = threadIdx.x;
  const size_t sn = (size_t)ne, N = (size_t)ne * Bs.nb;
  cd acc[Q9P_MAXNB];
  for (int b = 0; b < Q9P_MAXNB; ++b) acc[b] = mkc(0.0, 0.0);
  const cd ikb = mkc(-k * beta.y, k * beta.x);   // i k beta
  for (int p = 0; p < Q9_FAR; ++p) {
    const double* t = far_tab + (size_t)p * 7 * sn + f;
    __syncthreads();
    if (threadIdx.x == 0) {
      const double y[3] = {t[0], t[sn], t[2 * sn]};
      wave_setup(nt, y, k, &ws);
    }
    __syncthreads();
    if (q < B) {
      const double ny[3] = {t[3 * sn], t[4 * sn], t[5 * sn]};
      cd I, dI;
      wave_eval(nt, ws, q, ny, k, &I, &dI);
      const cd src = cadd(cmulr(cconj(dI), dsign), cmul(ikb, cconj(I)));
      double xi, eta, w, Nv[Q9P_MAXNB];
      q9_rule_point(R, 0, p, &xi, &eta, &w);
      q9p_shape(Bs, xi, eta, Nv, nullptr);
      for (int b = 0; b < Bs.nb; ++b) acc[b] = cadd(acc[b], cmulr(src, t[6 * sn] * Nv[b]));
    }
  }
  if (q < B)
    for (int b = 0; b < Bs.nb; ++b) V0[(size_t)q * N + (size_t)f * Bs.nb + b] = acc[b];
}

// U_0[i][q] at the collocation points; one CTA per element.
__global__ void k_l2p_table(const Elem* __restrict__ el, int n, int nt, double k, const double* __restrict__ centres,
                            cd* __restrict__ U0) {
  __shared__ WaveSetup ws;
  const int i = blockIdx.x;
  const Elem& E = el[i];
  const int B = (nt + 1) * (nt + 1);
  if (threadIdx.x == 0) {
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = E.c[d] - (centres ? centres[3 * i + d] : 0.0);
    wave_setup(nt, x, k, &ws);
  }
  __syncthreads();
  const int q = threadIdx.x;
  if (q >= B) return;
  cd I, dI;
  wave_eval(nt, ws, q, E.nrm, k, &I, &dI);
  int nn, m;
  q_to_nm(q, nn, m);
  // -(ik/4pi)(2n+1) [conj(I) + (i/k) conj(dI)]
  cd t = cadd(cconj(I), cmul(mkc(0.0, 1.0 / k), cconj(dI)));
  cd f = mkc(0.0, -k * (2 * nn + 1) * 0.25 / PI);
  U0[(size_t)i * B + q] = cmul(f, t);
}

// O_l^mu(d) for l <= 2 nt into shared memory, then K(d)[q][q'] for every
// pair.  One CTA per translation; block o is written at out + dest[o] B B
// (dest < 0: skipped).  regular: the same table with I_l = j_l Y_l in place
// of O_l = h_l Y_l (the coefficients of the regular addition theorem).
__global__ void k_m2l_blocks(int nt, double k, const double* __restrict__ dvecs, const int64_t* __restrict__ dest,
                             const double* __restrict__ W3, cd* __restrict__ out, int regular) {
  extern __shared__ double smem[];
  const int L = 2 * nt;
  cd* Osh = (cd*)smem;                               // (L+1)^2
  double* Psh = smem + 2 * (L + 1) * (L + 1);         // (L+1)^2
  __shared__ double jb[2 * MAX_NT + 2], yb[2 * MAX_NT + 2];
  __shared__ double ang[4];
  const int o = blockIdx.x;
  if (dest[o] < 0) return;
  const double d[3] = {dvecs[3 * o], dvecs[3 * o + 1], dvecs[3 * o + 2]};
  if (threadIdx.x == 0) {
    double r, ct, st, cp, sp;
    angles(d, r, ct, st, cp, sp);
    const double x = k * r;
    sph_bessel_j(L, x, jb);
    sph_bessel_y(L, x, yb);
    ferrers_tables(L, ct, st, Psh, nullptr);
    ang[0] = cp;
    ang[1] = sp;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (L + 1) * (L + 1); e += blockDim.x) {
    int l, m;
    q_to_nm(e, l, m);
    const cd ph = eimphi(m, ang[0], ang[1]);
    const double Y = ynorm(l, m) * Psh[l * (L + 1) + abs(m)];
    Osh[e] = cmul(mkc(jb[l], regular ? 0.0 : yb[l]), cmulr(ph, Y));
  }
  __syncthreads();
  const int B = (nt + 1) * (nt + 1);
  const int NL = nt + 1;
  cd* K = out + (size_t)dest[o] * B * B;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    const int q = e / B, qp = e - q * B;
    int n, m, n2, m2;
    q_to_nm(q, n, m);
    q_to_nm(qp, n2, m2);
    const int mu = m + m2;
    int lmin = max(abs(mu), abs(n - n2));
    if ((n + n2 - lmin) & 1) ++lmin;
    cd acc = mkc(0.0, 0.0);
    const double* w = W3 + (size_t)e * NL;
    for (int l = lmin, li = 0; l <= n + n2; l += 2, ++li) {
      const double c = w[li];
      if (c == 0.0) continue;
      // i^{n - n2 + l}
      const int p = ((n - n2 + l) % 4 + 4) % 4;
      const cd ip = p == 0 ? mkc(1, 0) : p == 1 ? mkc(0, 1) : p == 2 ? mkc(-1, 0) : mkc(0, -1);
      acc = cfma(cmulr(ip, c), Osh[l * (l + 1) + mu], acc);
    }
    const double sgn = (((m + m2) % 2) + 2) % 2 ? -1.0 : 1.0;
    K[e] = cmulr(acc, sgn * (2 * n2 + 1));
  }
}

// ----------------------------------------------------------- applications --
// Mom[r][c][q] = sum_j V_0[q][j] p[r][c][j]: one CTA per (r, c) column, p
// (float-float) in shared memory, one warp per coefficient row of V_0
// (float-float); Mom complex double.
__global__ void k_p2m_apply_ff(const float4* __restrict__ V0, int n, int B, const float4* __restrict__ p,
                               cd* __restrict__ Mom) {
  extern __shared__ float4 ps4[];
  const int64_t col = blockIdx.x;   // r * Nc + c
  const float4* src = p + col * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) ps4[j] = src[j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < B; q += nw) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4* row = V0 + (size_t)q * n;
    for (int j = lane; j < n; j += 32) ff_cmac(row[j], ps4[j], rh, rl, ih, il);
    ff_warp_sum(rh, rl);
    ff_warp_sum(ih, il);
    if (lane == 0) Mom[col * B + q] = mkc((double)rh + (double)rl, (double)ih + (double)il);
  }
}

// y[r][c][i] += sum_q U_0[i][q] Loc[r][c][q]: Loc (complex double) split into
// float-float in shared memory, one warp per row of U_0 (float-float).
__global__ void k_l2p_apply_ff(const float4* __restrict__ U0, int n, int B, const cd* __restrict__ Loc,
                               cd* __restrict__ y) {
  extern __shared__ float4 ls4[];
  const int64_t col = blockIdx.x;
  const cd* src = Loc + col * B;
  for (int q = threadIdx.x; q < B; q += blockDim.x) ls4[q] = split_ff(src[q]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4* row = U0 + (size_t)i * B;
    for (int q = lane; q < B; q += 32) ff_cmac(row[q], ls4[q], rh, rl, ih, il);
    ff_warp_sum(rh, rl);
    ff_warp_sum(ih, il);
    if (lane == 0) y[col * n + i] = cadd(y[col * n + i], mkc((double)rh + (double)rl, (double)ih + (double)il));
  }
}

// FP32 operators: V_0, U_0 and p complex FP32.
__global__ void k_p2m_apply_f32(const float2* __restrict__ V0, int n, int B, const float2* __restrict__ p,
                                cd* __restrict__ Mom) {
  extern __shared__ float2 ps2[];
  const int64_t col = blockIdx.x;
  const float2* src = p + col * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) ps2[j] = src[j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < B; q += nw) {
    float re = 0.f, im = 0.f;
    const float2* row = V0 + (size_t)q * n;
    for (int j = lane; j < n; j += 32) {
      const float2 a = row[j], b = ps2[j];
      re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
      im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) Mom[col * B + q] = mkc(re, im);
  }
}

__global__ void k_l2p_apply_f32(const float2* __restrict__ U0, int n, int B, const cd* __restrict__ Loc,
                                cd* __restrict__ y) {
  extern __shared__ float2 ls2[];
  const int64_t col = blockIdx.x;
  const cd* src = Loc + col * B;
  for (int q = threadIdx.x; q < B; q += blockDim.x) ls2[q] = make_float2((float)src[q].x, (float)src[q].y);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    float re = 0.f, im = 0.f;
    const float2* row = U0 + (size_t)i * B;
    for (int q = lane; q < B; q += 32) {
      const float2 a = row[q], b = ls2[q];
      re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
      im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) y[col * n + i] = cadd(y[col * n + i], mkc(re, im));
  }
}

// ------------------------------------------------------------- host side --
fmpb_status multipole_tables(const DeviceMesh& m, double k, cd beta, int nt, cd* V0, cd* U0, cudaStream_t st,
                             const double* centres, double dsign) {
  if (nt < 1 || nt > MAX_NT) {
    set_error("n_t must be 1..%d", MAX_NT);
    return FMPB_EINVAL;
  }
  if (m.nodes == 9 && m.q9_order > 0 && centres) {
    set_error("multipole_tables: per-element expansion centres take constant pressure on nine-node elements");
    return FMPB_EINVAL;
  }
  const int B = (nt + 1) * (nt + 1);
  const int threads = (B + 31) / 32 * 32;
  if (V0 && m.nodes == 9 && m.q9_order > 0)
    FMPB_LAUNCH("p2m_table_q9p", st, k_p2m_table_q9p<<<m.q9_ne, threads, 0, st>>>(m.q9_far, m.q9_ne, m.q9_order, nt, k, beta, m.q9r, dsign, V0));
  else if (V0 && m.nodes == 9)
    FMPB_LAUNCH("p2m_table_q9", st, k_p2m_table_q9<<<m.n, threads, 0, st>>>(m.q9_far, m.n, nt, k, beta, dsign, centres, V0));
  else if (V0)
    FMPB_LAUNCH("p2m_table", st, k_p2m_table<<<m.n, threads, 0, st>>>(m.el, m.n, nt, k, beta, m.qr, centres, V0));
  if (U0) FMPB_LAUNCH("l2p_table", st, k_l2p_table<<<m.n, threads, 0, st>>>(m.el, m.n, nt, k, centres, U0));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status wigner_table(int nt, double** W3out, cudaStream_t st) {
  const int B = (nt + 1) * (nt + 1);
  const size_t count = (size_t)B * B * (nt + 1);
  double* W3 = nullptr;
  FMPB_CUDA(cudaMallocAsync(&W3, sizeof(double) * count, st));
  FMPB_LAUNCH("wigner_table", st, k_wigner_table<<<std::min<size_t>(grid_for(count, 128), 152 * 8), 128, 0, st>>>(nt, W3));
  FMPB_CUDA(cudaGetLastError());
  *W3out = W3;
  return FMPB_OK;
}

fmpb_status m2l_blocks(int nt, double k, int n_d, const double* dvecs_host, const int64_t* dest_host, cd* out,
                       cudaStream_t st, bool regular) {
  if (nt < 1 || nt > MAX_NT) {
    set_error("n_t must be 1..%d", MAX_NT);
    return FMPB_EINVAL;
  }
  if (n_d <= 0) return FMPB_OK;
  double* W3 = nullptr;
  FMPB_TRY(wigner_table(nt, &W3, st));
  double* dd_ = nullptr;
  int64_t* dst = nullptr;
  FMPB_CUDA(cudaMallocAsync(&dd_, sizeof(double) * 3 * n_d, st));
  FMPB_CUDA(cudaMallocAsync(&dst, sizeof(int64_t) * n_d, st));
  FMPB_CUDA(cudaMemcpyAsync(dd_, dvecs_host, sizeof(double) * 3 * n_d, cudaMemcpyHostToDevice, st));
  FMPB_CUDA(cudaMemcpyAsync(dst, dest_host, sizeof(int64_t) * n_d, cudaMemcpyHostToDevice, st));
  const size_t smem = 3 * sizeof(double) * (2 * nt + 1) * (2 * nt + 1);
  FMPB_LAUNCH("m2l_blocks", st, k_m2l_blocks<<<n_d, 256, smem, st>>>(nt, k, dd_, dst, W3, out, regular ? 1 : 0));
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaFreeAsync(dd_, st));
  FMPB_CUDA(cudaFreeAsync(dst, st));
  FMPB_CUDA(cudaFreeAsync(W3, st));
  return FMPB_OK;
}

fmpb_status p2m_apply(const float4* V0, int n, int B, int64_t columns, const float4* p, cd* Mom, cudaStream_t st) {
  const size_t smem = sizeof(float4) * n;
  if (smem > 200 * 1024) {
    set_error("p2m_apply: %zu bytes of shared memory per block", smem);
    return FMPB_EINVAL;
  }
  FMPB_CUDA((smem_limit_once<k_p2m_apply_ff>(200 * 1024)));
  FMPB_LAUNCH("p2m_apply", st, k_p2m_apply_ff<<<(unsigned)columns, 256, smem, st>>>(V0, n, B, p, Mom));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status l2p_apply(const float4* U0, int n, int B, int64_t columns, const cd* Loc, cd* y, cudaStream_t st) {
  FMPB_LAUNCH("l2p_apply", st, k_l2p_apply_ff<<<(unsigned)columns, 256, sizeof(float4) * B, st>>>(U0, n, B, Loc, y));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

}  // namespace fmpb

namespace fmpb {

fmpb_status p2m_apply_f32(const float2* V0, int n, int B, int64_t columns, const float2* p, cd* Mom, cudaStream_t st) {
  FMPB_LAUNCH("p2m_apply_f32", st, k_p2m_apply_f32<<<(unsigned)columns, 256, sizeof(float2) * n, st>>>(V0, n, B, p, Mom));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status l2p_apply_f32(const float2* U0, int n, int B, int64_t columns, const cd* Loc, cd* y, cudaStream_t st) {
  FMPB_LAUNCH("l2p_apply_f32", st, k_l2p_apply_f32<<<(unsigned)columns, 256, sizeof(float2) * B, st>>>(U0, n, B, Loc, y));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

}  // namespace fmpb

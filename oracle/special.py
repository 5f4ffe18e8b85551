"""Special functions of the multipole expansion (Sec. 3.1, Eq. (Onm);
Appendix A, Eqs. (m2l), (wigner)).  Oracle code: test infrastructure only.

Conventions fixed here (the paper cites Liu 2009 and prints no normalisation):
  Y_n^m(theta, phi) = sqrt((n-m)!/(n+m)!) P_n^m(cos theta) e^{i m phi}
with P_n^m the Ferrers function WITHOUT the Condon-Shortley phase for m >= 0
and P_n^{-m} = (-1)^m (n-m)!/(n+m)! P_n^m (Rodrigues' formula), that is
  Y_n^m = s_m sqrt((n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{i m phi},
  s_m = (-1)^m for m < 0 and 1 otherwise.
Under this normalisation the printed expansion of G (Eq. (greenFMM)) is the
Gegenbauer addition theorem, sum_m Y_n^m(a) conj(Y_n^m(b)) = P_n(cos gamma),
and the Wigner-3j M2L of Eq. (m2l) holds (with the phase reading noted in
``oracle.fmm``).
O_n^m(x) = h_n^(1)(k|x|) Y_n^m(x/|x|), I_n^m(x) = j_n(k|x|) Y_n^m(x/|x|):
the printed Eq. (Onm) omits k, which the prefactor ik/4pi of Eq. (greenFMM)
requires.
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial, sqrt

import numpy as np
from scipy import special as sps


# ---------------------------------------------------------------- Bessel ----

def sph_jn(n: int, z):
    """Spherical Bessel function j_n (library primitive)."""
    return sps.spherical_jn(n, z)


def sph_jn_deriv(n: int, z):
    return sps.spherical_jn(n, z, derivative=True)


def sph_hn(n: int, z):
    """Spherical Hankel function of the first kind h_n = j_n + i y_n."""
    return sps.spherical_jn(n, z) + 1j * sps.spherical_yn(n, z)


def sph_hn_deriv(n: int, z):
    return sps.spherical_jn(n, z, derivative=True) + 1j * sps.spherical_yn(n, z, derivative=True)


# -------------------------------------------------------------- Legendre ----

def assoc_legendre_table(nmax: int, x):
    """P[n][m] for 0 <= m <= n <= nmax, no Condon-Shortley phase, by the
    three-term recurrence in n at fixed m started from
    P_m^m = (2m-1)!! (1-x^2)^{m/2},  P_{m+1}^m = (2m+1) x P_m^m."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    pmm = np.ones_like(x)
    for m in range(nmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        P[m][m] = pmm
        if m + 1 <= nmax:
            P[m + 1][m] = (2 * m + 1) * x * pmm
        for n in range(m + 2, nmax + 1):
            P[n][m] = ((2 * n - 1) * x * P[n - 1][m] - (n + m - 1) * P[n - 2][m]) / (n - m)
    return P


def legendre_over_sin_table(nmax: int, x):
    """Q[n][m] = P_n^m(x) / sqrt(1-x^2) for 1 <= m <= n <= nmax, computed by
    the same recurrence started from Q_m^m = (2m-1)!! (1-x^2)^{(m-1)/2}, which
    stays finite at the poles x = +-1."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    Q = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    qmm = np.ones_like(x)            # m = 1: (2*1-1)!! s^0 = 1
    for m in range(1, nmax + 1):
        if m > 1:
            qmm = qmm * (2 * m - 1) * s
        Q[m][m] = qmm
        if m + 1 <= nmax:
            Q[m + 1][m] = (2 * m + 1) * x * qmm
        for n in range(m + 2, nmax + 1):
            Q[n][m] = ((2 * n - 1) * x * Q[n - 1][m] - (n + m - 1) * Q[n - 2][m]) / (n - m)
    return Q


def norm_nm(n: int, m: int) -> float:
    """s_m sqrt((n-|m|)!/(n+|m|)!), the factor multiplying P_n^{|m|} e^{i m phi}."""
    sign = -1.0 if (m < 0 and (-m) % 2 == 1) else 1.0
    am = abs(m)
    return sign * sqrt(factorial(n - am) / factorial(n + am))


def coeff_index(n: int, m: int) -> int:
    """Flat index q = n(n+1) + m of coefficient (n, m), -n <= m <= n."""
    return n * (n + 1) + m


def coeff_list(nt: int):
    return [(n, m) for n in range(nt + 1) for m in range(-n, n + 1)]


def _angles(v):
    v = np.asarray(v, dtype=np.float64)
    r = np.linalg.norm(v, axis=-1)
    ct = np.where(r > 0, v[..., 2] / np.where(r > 0, r, 1.0), 1.0)
    ct = np.clip(ct, -1.0, 1.0)
    rho = np.hypot(v[..., 0], v[..., 1])
    # e^{i phi}; phi := 0 on the polar axis (every term there is continuous)
    eiphi = np.where(rho > 0, (v[..., 0] + 1j * v[..., 1]) / np.where(rho > 0, rho, 1.0), 1.0 + 0j)
    return r, ct, eiphi


def sph_harm_table(nmax: int, v):
    """Y[q] = Y_n^m(v/|v|) for every q = (n, m), n <= nmax."""
    r, ct, eiphi = _angles(v)
    P = assoc_legendre_table(nmax, ct)
    Y = []
    for n, m in coeff_list(nmax):
        Y.append(norm_nm(n, m) * P[n][abs(m)] * eiphi ** m)
    return np.array(Y)


def wave_table(nmax: int, v, k: float, kind: str):
    """I_n^m(v) (kind 'I', regular) or O_n^m(v) (kind 'O', outgoing) for all q."""
    r, ct, eiphi = _angles(v)
    P = assoc_legendre_table(nmax, ct)
    radial = [sph_jn(n, k * r) if kind == "I" else sph_hn(n, k * r) for n in range(nmax + 1)]
    return np.array([radial[n] * norm_nm(n, m) * P[n][abs(m)] * eiphi ** m
                     for n, m in coeff_list(nmax)])


def grad_regular_table(nmax: int, v, k: float):
    """Cartesian gradient of I_n^m at v, shape (B, ..., 3).

    grad(j_n(kr) Y) = k j_n'(kr) Y r_hat + (j_n(kr)/r) [dY/dtheta theta_hat
    + (i m / sin theta) Y phi_hat], with dP_n^m/dtheta and P_n^m/sin(theta)
    both evaluated through Q = P/sin(theta) so that the poles are regular;
    at r = 0 only n = 1 survives, with the limit grad(j_1(kr) Y_1^m)."""
    v = np.asarray(v, dtype=np.float64)
    r, ct, eiphi = _angles(v)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    P = assoc_legendre_table(nmax + 1, ct)
    Q = legendre_over_sin_table(nmax + 1, ct)
    cphi, sphi = eiphi.real, eiphi.imag
    rhat = np.stack([st * cphi, st * sphi, ct], axis=-1)
    that = np.stack([ct * cphi, ct * sphi, -st], axis=-1)
    phat = np.stack([-sphi, cphi, np.zeros_like(ct)], axis=-1)
    rs = np.where(r > 0, r, 1.0)
    out = []
    for n, m in coeff_list(nmax):
        am = abs(m)
        N = norm_nm(n, m)
        jn = sph_jn(n, k * r)
        jnp = sph_jn_deriv(n, k * r)
        if am == 0:
            # dP_n/dtheta = -sin(theta) P_n'(x), P_n' = n (x P_n - P_{n-1}) / (x^2 - 1)
            # written as -P_n^1 (no Condon-Shortley phase: P_n^1 = sin(theta) P_n')
            dP = -P[n][1] if n >= 1 else np.zeros_like(ct)
            phi_term = np.zeros_like(ct)
        else:
            # dP_n^m/dtheta = n x Q_n^m - (n+m) Q_{n-1}^m   (Q_{m-1}^m := 0)
            qn1 = Q[n - 1][am] if n - 1 >= am else np.zeros_like(ct)
            dP = n * ct * Q[n][am] - (n + am) * qn1
            phi_term = Q[n][am]
        e = eiphi ** m
        Yv = N * P[n][am] * e
        dYt = N * dP * e
        dYp = 1j * m * N * phi_term * e          # (1/sin theta) dY/dphi
        jn_over_r = np.where(r > 0, jn / rs, 0.0)
        g = (k * jnp * Yv)[..., None] * rhat + jn_over_r[..., None] * (dYt[..., None] * that + dYp[..., None] * phat)
        if n == 1:
            # r -> 0 limit: j_1(kr)/r -> k/3, j_1'(0) = 1/3
            at0 = r == 0
            if np.any(at0):
                g0 = _grad_degree1_at_origin(m, k)
                g = np.where(at0[..., None], g0, g)
        out.append(g)
    return np.array(out)


def _grad_degree1_at_origin(m: int, k: float):
    # j_1(kr) ~ kr/3: I_1^m ~ (k/3) r Y_1^m and r Y_1^m is linear:
    # r Y_1^0 = z, r Y_1^{1} = (x + i y)/sqrt 2, r Y_1^{-1} = -(x - i y)/sqrt 2
    if m == 0:
        return np.array([0, 0, k / 3.0], dtype=complex)
    s = norm_nm(1, m)
    return np.array([k / 3.0 * s, 1j * np.sign(m) * k / 3.0 * s, 0.0], dtype=complex)


# -------------------------------------------------------------- Wigner 3j --

@lru_cache(maxsize=None)
def _fact(n: int) -> int:
    return factorial(n)


@lru_cache(maxsize=None)
def wigner3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """Wigner 3j symbol by Racah's single-sum formula, summed exactly in
    rational arithmetic and rounded once (Shore & Menzel 1968, cited in the
    paper for Eq. (wigner))."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    tri = Fraction(_fact(j1 + j2 - j3) * _fact(j1 - j2 + j3) * _fact(-j1 + j2 + j3),
                   _fact(j1 + j2 + j3 + 1))
    pref = tri * _fact(j1 + m1) * _fact(j1 - m1) * _fact(j2 + m2) * _fact(j2 - m2) \
        * _fact(j3 + m3) * _fact(j3 - m3)
    tmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    tmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for t in range(tmin, tmax + 1):
        den = (_fact(t) * _fact(j3 - j2 + t + m1) * _fact(j3 - j1 + t - m2)
               * _fact(j1 + j2 - j3 - t) * _fact(j1 - t - m1) * _fact(j2 - t + m2))
        s += Fraction((-1) ** t, den)
    if s == 0:
        return 0.0
    sign = -1 if (j1 - j2 - m3) % 2 else 1
    # value = sign * s * sqrt(pref), evaluated as sign * sgn(s) * sqrt(s^2 pref)
    mag2 = s * s * pref
    val = sqrt(mag2.numerator) / sqrt(mag2.denominator) if mag2.numerator < 2 ** 1000 else float(mag2) ** 0.5
    return float(sign * (1 if s > 0 else -1) * val)

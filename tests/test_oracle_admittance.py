"""Pins of the oracle's admittance operator (Eq. (admittance) in Eq. (bm);
the matrix H - G Y of Eq. (matrixBEM) with a uniform normalised admittance):

* the analytic series for plane-wave scattering by a sphere with the same
  boundary condition, dp/dr = -i k beta p at r = a (the paper's normal points
  into the sphere), whose surface pressure is
  sum_n (2n+1) i^n [i / (ka)^2] / (h_n'(ka) + i beta h_n(ka)) P_n(cos theta)
  (Wronskian j_n h_n' - j_n' h_n = i / x^2); beta = 0 is the rigid series;
* the closed-form 1/r integral and the self single-layer integral (closed
  form + order-8 polar rule for the bounded remainder) against a brute-force
  collapsed rule of order 160 on the three children, where the Duffy map
  removes the 1/r singularity (the remaining integrand is smooth but sharply
  peaked for elongated triangles, hence the order);
* the adjoint double-layer kernel against central differences of G;
* beta = 0 reproducing the rigid blocks exactly;
* the FMM far field with the single-layer P2M term converging to the exact
  admittance blocks as n_t grows.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import bem, fmm
from oracle.special import sph_hn, sph_hn_deriv
from workloads import icosphere


def _impedance_sphere_surface(ka, beta, cos_theta, nmax=40):
    return sum((2 * n + 1) * 1j ** n * (1j / ka**2) / (sph_hn_deriv(n, ka) + 1j * beta * sph_hn(n, ka))
               * eval_legendre(n, cos_theta) for n in range(nmax))


@pytest.mark.parametrize("k,beta", [(2.0, 0.5 + 0.3j), (7.5, 1.0)])
def test_impedance_sphere_against_analytic_series(k, beta):
    errs = []
    for level in (2, 3):
        v, t = icosphere(level, 0.2)
        cell = bem.CellMesh(v, t)
        A = bem.toeplitz_block(cell, np.eye(3), (0, 0, 0), k, beta)
        b = bem.plane_wave_rhs(cell, np.eye(3), (1, 1, 1), k, [1.0, 0.0, 0.0])
        p = np.linalg.solve(A, b)
        ct = cell.centroid[:, 0] / np.linalg.norm(cell.centroid, axis=1)
        pa = _impedance_sphere_surface(k * 0.2, beta, ct)
        errs.append(np.linalg.norm(p - pa) / np.linalg.norm(pa))
    assert errs[0] < 0.03, errs
    assert errs[1] < 0.6 * errs[0], errs
    # the admittance matters: the rigid solution is far from this series
    rig = np.linalg.solve(bem.toeplitz_block(cell, np.eye(3), (0, 0, 0), k), b)
    assert np.linalg.norm(rig - pa) / np.linalg.norm(pa) > 5 * errs[1]


def _brute_self(tri, k, q=160):
    x = tri.mean(axis=0)
    out = 0.0 + 0.0j
    for e in range(3):
        pts, w = bem.collapsed_rule(x, tri[e], tri[(e + 1) % 3], q)
        out += np.sum(w * bem.kernel_slp(x, pts, k))
    return out


def test_closed_form_inverse_distance_integral():
    rng = np.random.default_rng(3)
    for _ in range(6):
        tri = rng.normal(size=(3, 3)) * 0.1
        x = tri.mean(axis=0)
        ref = 0.0
        for e in range(3):
            pts, w = bem.collapsed_rule(x, tri[e], tri[(e + 1) % 3], 160)
            ref += np.sum(w / np.linalg.norm(pts - x, axis=-1))
        assert abs(bem.inv_r_integral(tri, x) - ref) <= 1e-11 * ref


@pytest.mark.parametrize("k,tol", [(0.5, 1e-9), (6.0, 2e-7), (40.0, 1e-5)])
def test_self_single_layer_against_brute_force(k, tol):
    # The 1/r part is closed form (pinned above to 1e-11); the bounded
    # remainder (e^{ikr} - 1)/r uses the operator's order-8 polar rule, whose
    # error on these mesh elements (h about 0.12) grows with k h: about 4e-10,
    # 6e-8 and 3e-6 relative at k = 0.5, 6 and 40.
    v, t = icosphere(1, 0.2)
    for tri in np.asarray(v)[np.asarray(t)][:6]:
        ref = _brute_self(tri, k)
        assert abs(bem.self_slp(tri, k) - ref) <= tol * abs(ref)


def test_adjoint_double_layer_is_the_normal_derivative_of_g():
    rng = np.random.default_rng(4)
    for _ in range(5):
        x, y = rng.normal(size=3), rng.normal(size=3)
        nx = rng.normal(size=3)
        nx /= np.linalg.norm(nx)
        k, eps = 3.0, 1e-5
        fd = (bem.kernel_slp(x + eps * nx, y, k) - bem.kernel_slp(x - eps * nx, y, k)) / (2 * eps)
        got = bem.kernel_adlp(x, nx, y, k)
        assert abs(got - fd) <= 1e-8 * abs(got)


def test_zero_admittance_is_the_rigid_operator():
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    lat = np.diag([0.5, 0.5, 1.0])
    for d in [(0, 0, 0), (1, 0, 0), (2, -1, 0)]:
        a = bem.toeplitz_block(cell, lat, d, 3.0)
        b = bem.toeplitz_block(cell, lat, d, 3.0, 0.0)
        assert np.array_equal(a, b)
        c = bem.toeplitz_block(cell, lat, d, 3.0, 0.7)
        assert np.abs(c - a).max() > 1e-3 * np.abs(a).max()


def test_fmm_with_admittance_converges_to_exact_blocks():
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    lat = np.diag([0.6, 0.6, 1.0])
    counts, k, beta = (4, 1, 1), 4.0, 0.6 + 0.2j
    rng = np.random.default_rng(8)
    x = rng.normal(size=(1, 4 * cell.n)) + 1j * rng.normal(size=(1, 4 * cell.n))
    A = bem.dense_matrix(v, t, lat, counts, k, beta)
    exact = x @ A.T
    errs = [np.linalg.norm(fmm.fmm_matvec_explicit(cell, lat, counts, k, nt, x, beta=beta) - exact)
            / np.linalg.norm(exact) for nt in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6, errs


def _impedance_sphere_total(k, a, beta, pts, nmax=40):
    """Total pressure outside the sphere: sum_n (2n+1) i^n [j_n(kr) + A_n h_n(kr)] P_n(cos theta),
    A_n = -(j_n'(ka) + i beta j_n(ka)) / (h_n'(ka) + i beta h_n(ka)) from dp/dr = -i k beta p at r = a."""
    from oracle.special import sph_jn, sph_jn_deriv
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 0] / r
    ka = k * a
    out = np.zeros(len(pts), dtype=complex)
    for n in range(nmax):
        An = -(sph_jn_deriv(n, ka) + 1j * beta * sph_jn(n, ka)) / (sph_hn_deriv(n, ka) + 1j * beta * sph_hn(n, ka))
        out += (2 * n + 1) * 1j ** n * (sph_jn(n, k * r) + An * sph_hn(n, k * r)) * eval_legendre(n, ct)
    return out


@pytest.mark.parametrize("k,beta", [(3.0, 0.6 + 0.4j), (6.0, 1.0)])
def test_impedance_sphere_field_points_against_analytic_series(k, beta):
    # the exterior field of the collocation solution: the single layer that
    # the admittance adds (i k beta S p) is needed to reach the series
    v, t = icosphere(3, 0.2)
    cell = bem.CellMesh(v, t)
    A = bem.toeplitz_block(cell, np.eye(3), (0, 0, 0), k, beta)
    b = bem.plane_wave_rhs(cell, np.eye(3), (1, 1, 1), k, [1.0, 0.0, 0.0])
    p = np.linalg.solve(A, b)
    rng = np.random.default_rng(9)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = np.vstack([0.3 * dirs, 0.6 * dirs])
    ref = _impedance_sphere_total(k, 0.2, beta, pts)
    got = bem.field_points(v, t, np.eye(3), (1, 1, 1), k, p, pts, [1.0, 0.0, 0.0], beta=beta)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 0.01, err
    # dropping the admittance single layer misses the series by far more
    no_s = bem.field_points(v, t, np.eye(3), (1, 1, 1), k, p, pts, [1.0, 0.0, 0.0])
    assert np.linalg.norm(no_s - ref) / np.linalg.norm(ref) > 5 * err

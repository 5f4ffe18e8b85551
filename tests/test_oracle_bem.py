"""Pins of the oracle's Burton-Miller collocation operator (Sec. 2.1,
Eqs. (cbie), (hbie), (bm)) and its block Toeplitz form (Sec. 2.2): exact
polynomial integration, closed-form solid angles, Gauss flux and
hypersingular identities on closed meshes, the analytic rigid-sphere series,
and the statement that the PBEM matrix is an exact representation of the BEM
matrix (Sec. 4)."""
from math import factorial

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import bem
from oracle.special import sph_hn_deriv, sph_hn, sph_jn, sph_jn_deriv
from workloads import icosphere, cube, capped_cylinder


def test_collapsed_rule_integrates_polynomials_exactly():
    rng = np.random.default_rng(3)
    tri = rng.normal(size=(3, 3))
    e1, e2 = tri[1] - tri[0], tri[2] - tri[0]
    area = 0.5 * np.linalg.norm(np.cross(e1, e2))
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    for q in (3, 8):
        pts, w = bem.collapsed_rule(tri[0], tri[1], tri[2], q)
        rel = pts - tri[0]
        xi = np.linalg.solve(G, np.stack([rel @ e1, rel @ e2]))      # barycentric (xi1, xi2)
        for a in range(2 * q - 1):
            for b in range(2 * q - 1 - a):
                exact = 2 * area * factorial(a) * factorial(b) / factorial(a + b + 2)
                assert np.sum(w * xi[0] ** a * xi[1] ** b) == pytest.approx(exact, rel=1e-12)


def _solid_angle(x, tri):
    """van Oosterom & Strackee (1983): solid angle of a flat triangle seen from x."""
    R = tri - x
    r = np.linalg.norm(R, axis=1)
    num = R[0] @ np.cross(R[1], R[2])
    den = r[0] * r[1] * r[2] + (R[0] @ R[1]) * r[2] + (R[0] @ R[2]) * r[1] + (R[1] @ R[2]) * r[0]
    return 2.0 * np.arctan2(num, den)


@pytest.mark.parametrize("cls", [0, 1, 2])
def test_laplace_double_layer_equals_closed_form_solid_angle(cls):
    rng = np.random.default_rng(4)
    tri = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.03, 0.09, 0.0]])
    h = np.max(np.linalg.norm(tri - np.roll(tri, 1, axis=0), axis=1))
    cen = tri.mean(0)
    dist = {0: 5.0, 1: 2.5, 2: 1.0}[cls] * h
    tol = {0: 1e-5, 1: 1e-10, 2: 1e-4}[cls]
    for _ in range(5):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x = cen + dist * u
        assert bem.classify(x, cen, h) == cls
        D, _ = bem.pair_integrals(x[None], np.array([[0, 0, 1.0]]), tri[None], 0.0, cls)
        # dG0/dn_y integrated = -(solid angle)/(4 pi) with the element's own normal
        expect = -_solid_angle(x, tri) / (4 * np.pi)
        assert abs(D[0] - expect) <= tol * max(abs(expect), 1e-3)


@pytest.mark.parametrize("mesh", ["ico2", "cube", "cylinder"])
def test_gauss_flux_and_hypersingular_row_sums_on_closed_mesh(mesh):
    v, t = {"ico2": lambda: icosphere(2, 0.2), "cube": lambda: cube(0.3, 4),
            "cylinder": lambda: capped_cylinder(0.15, 0.6, 12, 6)}[mesh]()
    m = bem.CellMesh(v, t)
    D, H = bem.dh_block(m, m.v, 0.0, self_pairs=np.eye(m.n, dtype=bool))
    # Gauss: int dG0/dn_m = -1/2 at a smooth point of a closed surface (mesh normals
    # point out of the body), for every collocation point
    assert np.abs(D.sum(axis=1) + 0.5).max() < 1e-6
    # the double-layer potential of a constant density is piecewise constant, so
    # its normal derivative (finite-part row sum of the hypersingular kernel) is 0
    scale = np.abs(np.diag(H)).max()
    assert np.abs(H.sum(axis=1)).max() < 1e-4 * scale


def _rigid_sphere_surface(ka, cos_theta, nmax=40):
    # p(a, theta) = sum_n (2n+1) i^{n+1} P_n(cos theta) / ((ka)^2 h_n'(ka))
    return sum((2 * n + 1) * 1j ** (n + 1) * eval_legendre(n, cos_theta) / (ka**2 * sph_hn_deriv(n, ka))
               for n in range(nmax))


def _solve_single_sphere(level, k, a=0.2):
    v, t = icosphere(level, a)
    cell = bem.CellMesh(v, t)
    A = bem.toeplitz_block(cell, np.eye(3), (0, 0, 0), k)
    b = bem.plane_wave_rhs(cell, np.eye(3), (1, 1, 1), k, [1.0, 0.0, 0.0])
    return cell, v, t, np.linalg.solve(A, b)


@pytest.mark.parametrize("k", [2.0, 7.5])
def test_rigid_sphere_against_analytic_series(k):
    errs = []
    for level in (2, 3):
        cell, v, t, p = _solve_single_sphere(level, k)
        ct = cell.centroid[:, 0] / np.linalg.norm(cell.centroid, axis=1)
        pa = _rigid_sphere_surface(k * 0.2, ct)
        errs.append(np.linalg.norm(p - pa) / np.linalg.norm(pa))
    assert errs[0] < 0.03
    assert errs[1] < 0.6 * errs[0]


def test_field_points_against_analytic_exterior_field():
    k, a = 2.0, 0.2
    cell, v, t, p = _solve_single_sphere(2, k, a)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(12, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pts = u * np.array([0.3, 0.45, 0.8] * 4)[:, None]
    out = bem.field_points(v, t, np.eye(3), (1, 1, 1), k, p, pts, [1.0, 0, 0])
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 0] / r
    ka = k * a
    exact = sum((2 * n + 1) * 1j**n * (sph_jn(n, k * r) - sph_jn_deriv(n, ka) / sph_hn_deriv(n, ka) * sph_hn(n, k * r))
                * eval_legendre(n, ct) for n in range(40))
    assert np.abs(out - exact).max() < 0.01 * np.abs(exact).max()


def test_pbem_blocks_are_an_exact_representation_of_the_dense_matrix():
    v, t = icosphere(1, 0.2)
    lattice = np.diag([0.5, 0.6, 1.0])
    counts = (3, 2, 1)
    k = 3.0
    A = bem.dense_matrix(v, t, lattice, counts, k)
    cell = bem.CellMesh(v, t)
    cells = bem.lattice_cells(counts)
    n = cell.n
    blocks = {d: bem.toeplitz_block(cell, lattice, d, k) for d in bem.all_offsets(counts)}
    for ci, c in enumerate(cells):
        for cj, cp in enumerate(cells):
            delta = tuple(x - y for x, y in zip(c, cp))
            blk = A[ci * n:(ci + 1) * n, cj * n:(cj + 1) * n]
            assert np.abs(blk - blocks[delta]).max() <= 1e-13 * np.abs(blk).max()
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, A.shape[0])) + 1j * rng.normal(size=(2, A.shape[0]))
    y = bem.toeplitz_matvec(blocks, counts, x)
    assert np.linalg.norm(y - x @ A.T) <= 1e-13 * np.linalg.norm(y)

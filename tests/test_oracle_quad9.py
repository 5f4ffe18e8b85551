"""Pins of the oracle's nine-node quadratic quadrilateral operator (the
paper's element family, constant pressure collocated at the element centre):

* shape functions: partition of unity, nodal interpolation, derivatives
  against central differences;
* the flux and hypersingular identities on a closed surface (row sums of D
  equal -1/2 and of H vanish as k -> 0), which hold exactly for the closed
  surface the curved elements form and so test the self terms (the
  hypersingular finite part) to quadrature accuracy; a wrong leading Laurent
  coefficient, finite-part sign or polar Jacobian fails them by orders of
  magnitude;
* on a flat element the finite part equals the flat-polygon closed form
  (edge sum of the r^-3 finite part plus the bounded remainder), and the
  single layer the closed-form 1/r integral plus its remainder;
* the analytic rigid-sphere series: error falling with refinement, and fewer
  unknowns than flat triangles for the same accuracy.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import bem, quad9
from oracle.special import sph_hn_deriv
from workloads import quad9_sphere, icosphere


def test_shape_functions():
    rng = np.random.default_rng(1)
    xi, eta = rng.uniform(-1, 1, 7), rng.uniform(-1, 1, 7)
    N, Nx, Ne, Nxx, Nxe, Nee = quad9.shape(xi, eta)
    assert np.allclose(N.sum(axis=0), 1.0, atol=1e-14)
    grid = [(-1.0, 0.0, 1.0)[i] for i in range(3)]
    for j in range(3):
        for i in range(3):
            Ni = quad9.shape(np.array([grid[i]]), np.array([grid[j]]))[0][:, 0]
            assert np.allclose(Ni, np.eye(9)[3 * j + i], atol=1e-14)
    h = 1e-6
    for d, (a, b) in ((Nx, (h, 0)), (Ne, (0, h))):
        fd = (quad9.shape(xi + a, eta + b)[0] - quad9.shape(xi - a, eta - b)[0]) / (2 * h)
        assert np.abs(fd - d).max() < 1e-8
    fd = (quad9.shape(xi + h, eta)[1] - quad9.shape(xi - h, eta)[1]) / (2 * h)
    assert np.abs(fd - Nxx).max() < 1e-7
    fd = (quad9.shape(xi, eta + h)[1] - quad9.shape(xi, eta - h)[1]) / (2 * h)
    assert np.abs(fd - Nxe).max() < 1e-7


@pytest.mark.parametrize("m", [2, 3])
def test_closed_surface_identities(m):
    nodes, el = quad9_sphere(m, 0.2)
    mesh = quad9.Q9Mesh(nodes, el)
    D, H, S, K = quad9.dhsk_block(mesh, mesh.Y, 1e-3, self_pairs=np.eye(mesh.n, dtype=bool))
    assert np.abs(D.sum(axis=1) + 0.5).max() < 1e-7
    assert np.abs(H.sum(axis=1)).max() < 1e-6 * np.abs(H).max()


def _flat_q9(a, b, c, d):
    """Nine nodes of the flat (bilinear) quadrilateral with corners a, b, c, d
    (counter-clockwise), node (i, j) at 3 j + i."""
    Y = []
    for eta in (-1.0, 0.0, 1.0):
        for xi in (-1.0, 0.0, 1.0):
            w = np.array([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta), (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)]) / 4
            Y.append(w[0] * a + w[1] * b + w[2] * c + w[3] * d)
    return np.array(Y)


@pytest.mark.parametrize("k", [0.5, 4.0])
def test_flat_element_self_terms_equal_the_closed_forms(k):
    corners = [np.array(p) for p in ([0.0, 0.0, 0.0], [0.11, 0.01, 0.0], [0.13, 0.09, 0.0], [-0.01, 0.1, 0.0])]
    Y = _flat_q9(*corners)
    D, H, S, K = quad9.self_integrals(Y, k)
    x = quad9.geometry(Y, 0.0, 0.0)[0]
    fp = invr = 0.0
    for e in range(4):
        a, b = corners[e], corners[(e + 1) % 4]
        eh = (b - a) / np.linalg.norm(b - a)
        ta, tb = np.dot(a - x, eh), np.dot(b - x, eh)
        he = np.linalg.norm((a - x) - ta * eh)
        fp -= (tb / np.linalg.norm(b - x) - ta / np.linalg.norm(a - x)) / he
        invr += he * np.log((tb + np.linalg.norm(b - x)) / (ta + np.linalg.norm(a - x)))
    rem_h = rem_s = 0.0
    for e in range(4):
        pts, w = bem.collapsed_rule(x, corners[e], corners[(e + 1) % 4], 40)
        r = np.linalg.norm(pts - x, axis=-1)
        rem_h += np.sum(w * (np.exp(1j * k * r) * (1 - 1j * k * r) - 1) / r ** 3)
        rem_s += np.sum(w * (np.exp(1j * k * r) - 1) / r)
    assert abs(D) < 1e-14 and abs(K) < 1e-14
    Href = (fp + rem_h) / (4 * np.pi)
    Sref = (invr + rem_s) / (4 * np.pi)
    assert abs(H - Href) < 1e-9 * abs(Href)
    assert abs(S - Sref) < 1e-9 * abs(Sref)


def _series(ka, ct, nmax=40):
    return sum((2 * n + 1) * 1j ** n * (1j / ka ** 2) / sph_hn_deriv(n, ka) * eval_legendre(n, ct)
               for n in range(nmax))


def test_rigid_sphere_against_the_analytic_series():
    k, a = 2.0, 0.2
    errs = []
    for m in (2, 4):
        nodes, el = quad9_sphere(m, a)
        mesh = quad9.Q9Mesh(nodes, el)
        p = np.linalg.solve(quad9.dense_matrix(nodes, el, k), quad9.plane_wave_rhs(mesh, k, [1.0, 0.0, 0.0]))
        ct = mesh.centroid[:, 0] / np.linalg.norm(mesh.centroid, axis=1)
        pa = _series(k * a, ct)
        errs.append(np.linalg.norm(p - pa) / np.linalg.norm(pa))
    assert errs[1] < 0.3 * errs[0] and errs[1] < 6e-3, errs
    # flat triangles need more unknowns for the same accuracy (320 against 96)
    v, t = icosphere(2, a)
    cell = bem.CellMesh(v, t)
    pt = np.linalg.solve(bem.dense_matrix(v, t, np.eye(3), (1, 1, 1), k),
                         bem.plane_wave_rhs(cell, np.eye(3), (1, 1, 1), k, [1.0, 0.0, 0.0]))
    ct = cell.centroid[:, 0] / np.linalg.norm(cell.centroid, axis=1)
    et = np.linalg.norm(pt - _series(k * a, ct)) / np.linalg.norm(_series(k * a, ct))
    assert errs[1] < 1.1 * et


def test_periodic_blocks_equal_the_dense_matrix_of_the_array():
    nodes, el = quad9_sphere(2, 0.2)
    cell = quad9.Q9Mesh(nodes, el)
    L, counts, k = np.diag([0.5, 0.55, 1.0]), (2, 2, 1), 3.0
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, float) @ L for c in cells])
    allE = np.concatenate([el + i * len(nodes) for i in range(len(cells))])
    A = quad9.dense_matrix(allN, allE, k, 0.3 + 0.2j)
    n = cell.n
    for ci, c in enumerate(cells):
        for cj, cp in enumerate(cells):
            d = tuple(a - b for a, b in zip(c, cp))
            T = quad9.toeplitz_block(cell, L, d, k, 0.3 + 0.2j)
            # the translated node coordinates differ by rounding, which the
            # finite part of the self term amplifies to about 1e-11
            assert np.abs(A[ci * n:(ci + 1) * n, cj * n:(cj + 1) * n] - T).max() <= 1e-10 * np.abs(T).max()


@pytest.mark.parametrize("beta", [0.0, 0.3 + 0.2j])
def test_fmm_product_on_q9_cells_tends_to_the_exact_operator(beta):
    # the far cells' blocks use the same 4 x 4 rule as the P2M table, so the
    # FMPBEM product converges to the exact block Toeplitz product to
    # rounding; the centre's normal in place of each point's stalls it at
    # 6e-5, a missing conjugate or admittance term far higher
    nodes, el = quad9_sphere(2, 0.2)
    cell = quad9.Q9Mesh(nodes, el)
    L, counts, k = np.eye(3), (4, 1, 1), 2.0
    blocks = {d: quad9.toeplitz_block(cell, L, d, k, beta) for d in bem.all_offsets(counts)}
    rng = np.random.default_rng(7)
    p = rng.standard_normal(cell.n * 4) + 1j * rng.standard_normal(cell.n * 4)
    y_exact = bem.toeplitz_matvec(blocks, counts, p)[0]
    errs = []
    for nt in (2, 4, 6, 8, 10, 12):
        y = quad9.fmm_matvec_explicit(cell, L, counts, k, nt, p, beta)[0]
        errs.append(np.linalg.norm(y - y_exact) / np.linalg.norm(y_exact))
    assert all(b < 0.05 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-13, errs


def test_fmm2_near_block_on_q9_cells_tends_to_the_exact_block():
    # the multilevel near field of a Q9 cell (octree of the element centres,
    # leaf P2M over the far rule with each point's normal): 372 translated box
    # pairs at three levels; the centre normal in the leaf P2M stalls at 1e-4
    nodes, el = quad9_sphere(3, 0.2)
    mesh = quad9.Q9Mesh(nodes, el)
    L = np.diag([0.6, 0.6, 1.0])
    S = quad9.toeplitz_block(mesh, L, (0, 0, 0), 3.0, 0.3j)
    errs = [np.linalg.norm(quad9.fmm2_near_block(mesh, L, (0, 0, 0), 3.0, ntn, 3, 0.3j) - S) / np.linalg.norm(S)
            for ntn in (4, 8)]
    assert errs[1] < 0.01 * errs[0] and errs[1] < 1e-6, errs

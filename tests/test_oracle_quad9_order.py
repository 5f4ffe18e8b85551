"""Pins of the oracle's nine-node quadrilaterals with discontinuous pressure of
order 0, 1 and 2 (the paper's variable-order pressure):

* shape functions: nodal interpolation, partition of unity, reproduction of
  the bilinear (order 1) and eight-node serendipity (order 2) polynomial
  spaces, gradients against central differences;
* order 0 is the constant element of quad9.py, entry for entry;
* the closed-surface flux and hypersingular row sums (the constant density);
* on a flat element with a non-affine map, the finite part of each shape
  function at each off-centre node equals an independent decomposition:
  N_b(x) times the polygon closed form, grad N_b(x) . (the principal value
  of (y - x)/r^3, an edge sum of int ds/r), and the bounded remainder by a
  96-point collapsed rule in physical space;
* Green's identities for a linear harmonic field on a closed Q9 sphere
  (non-constant densities on curved elements): the representation error of
  order 1 and the hypersingular error of order 2 fall with refinement at
  their orders; dropping the gradient term of the Laurent coefficient leaves
  the row sums intact but stalls the hypersingular identity near 0.3;
* the analytic rigid sphere, where order 2 is more accurate per unknown;
* the periodic blocks equal the dense matrix of the whole array.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import bem, quad9, quad9_order as qo
from oracle.special import sph_hn_deriv
from workloads import quad9_sphere


@pytest.mark.parametrize("order", [0, 1, 2])
def test_pressure_basis(order):
    b = qo.PressureBasis(order)
    assert b.nb == (1, 4, 8)[order]
    N, _ = b.eval(b.nodes[:, 0], b.nodes[:, 1])
    assert np.allclose(N, np.eye(b.nb), atol=1e-14)
    rng = np.random.default_rng(3)
    xi, eta = rng.uniform(-1, 1, 9), rng.uniform(-1, 1, 9)
    N, G = b.eval(xi, eta)
    assert np.allclose(N.sum(axis=0), 1.0, atol=1e-14)
    # reproduction of the element's polynomial space from nodal values
    space = {0: [lambda x, y: 1 + 0 * x],
             1: [lambda x, y: 1 + 0 * x, lambda x, y: x, lambda x, y: y, lambda x, y: x * y],
             2: [lambda x, y: 1 + 0 * x, lambda x, y: x, lambda x, y: y, lambda x, y: x * x, lambda x, y: x * y,
                 lambda x, y: y * y, lambda x, y: x * x * y, lambda x, y: x * y * y]}[order]
    for f in space:
        assert np.allclose(f(b.nodes[:, 0], b.nodes[:, 1]) @ N, f(xi, eta), atol=1e-13)
    h = 1e-6
    for d, (a, c) in enumerate(((h, 0.0), (0.0, h))):
        fd = (b.eval(xi + a, eta + c)[0] - b.eval(xi - a, eta - c)[0]) / (2 * h)
        assert np.abs(fd - G[:, d]).max() < 1e-8


def test_order_zero_is_the_constant_element():
    nodes, el = quad9_sphere(2, 0.2)
    A0 = qo.dense_matrix(nodes, el, 0, 3.0, 0.3 + 0.2j)
    Aq = quad9.dense_matrix(nodes, el, 3.0, 0.3 + 0.2j)
    assert np.abs(A0 - Aq).max() <= 1e-14 * np.abs(Aq).max()


@pytest.mark.parametrize("order", [1, 2])
def test_closed_surface_identities(order):
    nodes, el = quad9_sphere(2, 0.2)
    mesh = qo.OrderMesh(nodes, el, order)
    D, H, S, K = qo.dhsk_block(mesh, mesh.geo.Y, 1e-3, self_same=True)
    assert np.abs(D.sum(axis=1) + 0.5).max() < 5e-8
    assert np.abs(H.sum(axis=1)).max() < 1e-8 * np.abs(H).max()


def _flat_q9(a, b, c, d):
    Y = []
    for eta in (-1.0, 0.0, 1.0):
        for xi in (-1.0, 0.0, 1.0):
            w = np.array([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta), (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)]) / 4
            Y.append(w[0] * a + w[1] * b + w[2] * c + w[3] * d)
    return np.array(Y)


def _inverse_map(Y, pts):
    """(xi, eta) of points of a flat element by Newton's method."""
    xi, eta = np.zeros(len(pts)), np.zeros(len(pts))
    for _ in range(30):
        y, yx, ye = quad9.geometry(Y, xi, eta)[:3]
        M = np.stack([yx, ye], axis=-1)
        step = np.linalg.solve(np.einsum("pdi,pdj->pij", M, M),
                               np.einsum("pdi,pd->pi", M, pts - y)[..., None])[..., 0]
        xi, eta = xi + step[:, 0], eta + step[:, 1]
    return xi, eta


@pytest.mark.parametrize("order,k", [(1, 0.5), (2, 4.0)])
def test_flat_element_finite_part_with_the_gradient_term(order, k):
    corners = [np.array(p) for p in ([0.0, 0.0, 0.0], [0.11, 0.01, 0.0], [0.13, 0.09, 0.0], [-0.01, 0.1, 0.0])]
    Y = _flat_q9(*corners)
    basis = qo.PressureBasis(order)
    nrm = np.cross(corners[1] - corners[0], corners[2] - corners[0])
    nrm /= np.linalg.norm(nrm)
    for a in range(basis.nb):
        D, H, S, K = qo.self_integrals(Y, basis, a, k)
        xa, ea = basis.nodes[a]
        x, yx, ye = quad9.geometry(Y, xa, ea)[:3]
        N0, G0 = basis.eval(np.array(xa), np.array(ea))
        N0, G0 = N0.reshape(-1), G0.reshape(-1, 2)
        M = np.stack([yx, ye], axis=-1)
        gy = (M @ np.linalg.inv(M.T @ M) @ G0.T).T          # in-plane gradients of N_b at x
        fp, pv, invr = 0.0, np.zeros(3), 0.0
        for e in range(4):
            p, q = corners[e], corners[(e + 1) % 4]
            eh = (q - p) / np.linalg.norm(q - p)
            ta, tb = np.dot(p - x, eh), np.dot(q - x, eh)
            he = np.linalg.norm((p - x) - ta * eh)
            ra, rb = np.linalg.norm(p - x), np.linalg.norm(q - x)
            fp -= (tb / rb - ta / ra) / he                   # finite part of int r^-3
            line = np.log((tb + rb) / (ta + ra))             # int ds / r along the edge
            pv -= np.cross(eh, nrm) * line                   # PV int (y - x) / r^3 = -sum nu int ds/r
            invr += he * line                                # int 1/r
        rem_h = np.zeros(basis.nb, dtype=complex)
        rem_s = np.zeros(basis.nb, dtype=complex)
        for e in range(4):
            pts, w = bem.collapsed_rule(x, corners[e], corners[(e + 1) % 4], 96)
            Nb, _ = basis.eval(*_inverse_map(Y, pts))
            r = np.linalg.norm(pts - x, axis=-1)
            lin = N0[:, None] + gy @ (pts - x).T
            rem_h += (Nb - lin) @ (w / r ** 3) + Nb @ (w * (np.exp(1j * k * r) * (1 - 1j * k * r) - 1) / r ** 3)
            rem_s += (Nb - N0[:, None]) @ (w / r) + Nb @ (w * (np.exp(1j * k * r) - 1) / r)
        Href = (N0 * fp + gy @ pv + rem_h) / (4 * np.pi)
        Sref = (N0 * invr + rem_s) / (4 * np.pi)
        assert np.abs(D).max() < 1e-14 and np.abs(K).max() < 1e-14
        assert np.abs(H - Href).max() < 2e-9 * np.abs(Href).max(), a
        # S integrates directly (no subtraction): 24 nodes per direction
        # leave about 1e-8 of quadrature error on the thin triangle towards
        # the nearest side
        assert np.abs(S - Sref).max() < 5e-8 * np.abs(Sref).max(), a


def _green_errors(order, m, k=1e-4):
    nodes, el = quad9_sphere(m, 0.2)
    mesh = qo.OrderMesh(nodes, el, order)
    D, H, S, K = qo.dhsk_block(mesh, mesh.geo.Y, k, self_same=True)
    g = np.array([1.0, 0.5, -0.3])
    u, dudn = mesh.points @ g, mesh.normals @ g
    rep = D @ u - S @ dudn + 0.5 * u            # -u/2 = D u - S du/dn
    hyp = H @ u - K @ dudn + 0.5 * dudn         # -(du/dn_x)/2 = H u - K du/dn
    return np.abs(rep).max() / np.abs(u).max(), np.abs(hyp).max() / np.abs(dudn).max()


def test_green_identities_with_a_linear_harmonic_field():
    r2, _ = _green_errors(1, 2)
    r3, _ = _green_errors(1, 3)
    assert r2 < 2e-3 and r3 < 0.4 * r2              # O(h^3) for the bilinear density
    _, h2 = _green_errors(2, 2)
    _, h3 = _green_errors(2, 3)
    assert h2 < 6e-3 and h3 < 0.45 * h2             # O(h^2): the quadratic density through H


def _series(ka, ct, nmax=40):
    return sum((2 * n + 1) * 1j ** n * (1j / ka ** 2) / sph_hn_deriv(n, ka) * eval_legendre(n, ct)
               for n in range(nmax))


def _sphere_error(order, m, k=2.0, a=0.2):
    nodes, el = quad9_sphere(m, a)
    mesh = qo.OrderMesh(nodes, el, order)
    p = np.linalg.solve(qo.dense_matrix(nodes, el, order, k), qo.plane_wave_rhs(mesh, k, [1.0, 0.0, 0.0]))
    pa = _series(k * a, mesh.points[:, 0] / np.linalg.norm(mesh.points, axis=1))
    return np.linalg.norm(p - pa) / np.linalg.norm(pa), len(p)


def test_rigid_sphere_quadratic_pressure_per_unknown():
    e2, n2 = _sphere_error(2, 1)       # 6 elements x 8 nodes
    e0, n0 = _sphere_error(0, 3)       # 54 elements x 1 node
    assert n2 < n0 and e2 < 0.5 * e0 and e2 < 4e-3, (e2, e0)


def test_periodic_blocks_equal_the_dense_matrix_of_the_array():
    nodes, el = quad9_sphere(1, 0.2)
    cell = qo.OrderMesh(nodes, el, 1)
    L, counts, k, beta = np.diag([0.5, 0.55, 1.0]), (2, 1, 1), 3.0, 0.3 + 0.2j
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, float) @ L for c in cells])
    allE = np.concatenate([el + i * len(nodes) for i in range(len(cells))])
    A = qo.dense_matrix(allN, allE, 1, k, beta)
    n = cell.n * cell.nb
    for ci, c in enumerate(cells):
        for cj, cp in enumerate(cells):
            d = tuple(x - y for x, y in zip(c, cp))
            T = qo.toeplitz_block(cell, L, d, k, beta)
            # translated node coordinates differ by rounding, which the
            # finite part amplifies by (rho_hat / rho_min)^2 (the thin
            # triangles of off-centre nodes reach rho_min of about 5e-4)
            assert np.abs(A[ci * n:(ci + 1) * n, cj * n:(cj + 1) * n] - T).max() <= 5e-9 * np.abs(T).max()


@pytest.mark.parametrize("order,beta", [(1, 0.0), (2, 0.3 + 0.2j)])
def test_fmm_product_tends_to_the_exact_operator(order, beta):
    # the far cells' blocks use the same 4 x 4 rule as the P2M table, so the
    # FMPBEM product converges to the exact block Toeplitz product to
    # rounding; shape functions taken at the element centre instead of each
    # point stall it at 1e-3
    nodes, el = quad9_sphere(1, 0.2)
    cell = qo.OrderMesh(nodes, el, order)
    L, counts, k = np.eye(3), (4, 1, 1), 2.0
    blocks = {d: qo.toeplitz_block(cell, L, d, k, beta) for d in bem.all_offsets(counts)}
    rng = np.random.default_rng(7)
    N = cell.n * cell.nb * 4
    p = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y_exact = bem.toeplitz_matvec(blocks, counts, p)[0]
    errs = [np.linalg.norm(qo.fmm_matvec_explicit(cell, L, counts, k, nt, p, beta)[0] - y_exact)
            / np.linalg.norm(y_exact) for nt in (4, 8, 12)]
    assert errs[1] < 1e-3 * errs[0] and errs[2] < 1e-13, errs


def test_order_zero_p2m_is_the_constant_elements():
    nodes, el = quad9_sphere(1, 0.2)
    V = qo.p2m_table(qo.OrderMesh(nodes, el, 0), 2.0, 6, 0.3j)
    Vq = quad9.p2m_table(quad9.Q9Mesh(nodes, el), 2.0, 6, 0.3j)
    assert np.abs(V - Vq).max() <= 1e-14 * np.abs(Vq).max()


def _impedance_sphere_total(k, a, beta, pts, nmax=40):
    """sum_n (2n+1) i^n [j_n(kr) + A_n h_n(kr)] P_n(cos theta) outside the sphere,
    A_n = -(j_n'(ka) + i beta j_n(ka)) / (h_n'(ka) + i beta h_n(ka)) (dp/dr = -i k beta p at r = a)."""
    from oracle.special import sph_jn, sph_jn_deriv, sph_hn
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 0] / r
    ka = k * a
    out = np.zeros(len(pts), dtype=complex)
    for n in range(nmax):
        An = -(sph_jn_deriv(n, ka) + 1j * beta * sph_jn(n, ka)) / (sph_hn_deriv(n, ka) + 1j * beta * sph_hn(n, ka))
        out += (2 * n + 1) * 1j ** n * (sph_jn(n, k * r) + An * sph_hn(n, k * r)) * eval_legendre(n, ct)
    return out


@pytest.mark.parametrize("order,m,beta", [(1, 2, 0.0), (2, 1, 0.6 + 0.4j)])
def test_field_points_against_the_analytic_sphere(order, m, beta):
    k = 3.0
    nodes, el = quad9_sphere(m, 0.2)
    mesh = qo.OrderMesh(nodes, el, order)
    p = np.linalg.solve(qo.toeplitz_block(mesh, np.eye(3), (0, 0, 0), k, beta),
                        qo.plane_wave_rhs(mesh, k, [1.0, 0.0, 0.0]))
    rng = np.random.default_rng(9)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = np.vstack([0.3 * dirs, 0.6 * dirs])
    ref = _impedance_sphere_total(k, 0.2, beta, pts)
    got = qo.field_points(nodes, el, order, np.eye(3), (1, 1, 1), k, p, pts, [1.0, 0.0, 0.0], beta=beta)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 5e-3, err
    if beta != 0:
        # the admittance single layer is needed to reach the series
        no_s = qo.field_points(nodes, el, order, np.eye(3), (1, 1, 1), k, p, pts, [1.0, 0.0, 0.0])
        assert np.linalg.norm(no_s - ref) / np.linalg.norm(ref) > 5 * err


@pytest.mark.parametrize("order,m", [(0, 2), (1, 2), (2, 1)])
def test_halfspace_image_method(order, m):
    # a sphere above a rigid plane (R_p = 1) has the surface solution of the
    # sphere and its mirror image in full space under the incident wave and
    # its image; the mirrored sphere of the full-space problem is wound
    # outward by reversing xi, the image part keeps the node order and
    # negates the terms linear in n_y (leaving that negation out moves the
    # solution by 7e-2)
    from oracle import halfspace
    k, plane, d = 3.0, halfspace.Plane(2, -0.3, 1.0), np.array([0.6, 0.0, -0.8])
    nodes, el = quad9_sphere(m, 0.2)
    mesh = qo.OrderMesh(nodes, el, order)
    Ah = (qo.toeplitz_block(mesh, np.eye(3), (0, 0, 0), k)
          + qo.image_block(mesh, np.eye(3), (1, 1, 1), plane, (0, 0, 0), k))
    ph = np.linalg.solve(Ah, qo.incident_with_image(mesh, k, d, plane))
    rev = np.array([2, 1, 0, 5, 4, 3, 8, 7, 6])
    N2 = np.concatenate([nodes, plane.mirror(nodes)])
    E2 = np.concatenate([el, el[:, rev] + len(nodes)])
    m2 = qo.OrderMesh(N2, E2, order)
    e1, e2 = np.exp(1j * k * (m2.points @ d)), np.exp(1j * k * (plane.mirror(m2.points) @ d))
    b2 = e1 + e2 + bem.coupling(k) * 1j * k * ((m2.normals @ d) * e1 + (plane.reflect(m2.normals) @ d) * e2)
    p2 = np.linalg.solve(qo.dense_matrix(N2, E2, order, k), b2)
    assert np.linalg.norm(ph - p2[:len(ph)]) / np.linalg.norm(ph) < 1e-9


@pytest.mark.parametrize("counts,L", [((2, 1, 2), np.diag([0.5, 1.0, 0.45])), ((3, 2, 1), np.diag([0.5, 0.45, 1.0]))])
def test_halfspace_structured_product_equals_the_dense_matrix(counts, L):
    # Toeplitz part plus the image part (block Hankel along a perpendicular
    # axis, applied to the cell-reversed vector) against the plain matrix
    from oracle import halfspace
    from workloads import random_complex_vectors
    plane = halfspace.Plane(2, -0.3, 1.0)
    nodes, el = quad9_sphere(1, 0.2)
    A = qo.dense_matrix_halfspace(nodes, el, 1, L, counts, 3.0, plane, 0.3 + 0.2j)
    x = random_complex_vectors(5, 1, A.shape[0])
    y = qo.structured_matvec_halfspace(qo.OrderMesh(nodes, el, 1), L, counts, 3.0, plane, x, 0.3 + 0.2j)
    assert np.linalg.norm(y - x @ A.T) / np.linalg.norm(x @ A.T) < 5e-9


@pytest.mark.parametrize("order,m", [(0, 2), (2, 1)])
def test_halfspace_field_points_image_method(order, m):
    # the half-space field of a sphere above a rigid plane equals the
    # full-space field of the sphere pair under the wave and its image
    from oracle import halfspace
    k, plane, d = 3.0, halfspace.Plane(2, -0.3, 1.0), np.array([0.6, 0.0, -0.8])
    nodes, el = quad9_sphere(m, 0.2)
    mesh = qo.OrderMesh(nodes, el, order)
    Ah = (qo.toeplitz_block(mesh, np.eye(3), (0, 0, 0), k)
          + qo.image_block(mesh, np.eye(3), (1, 1, 1), plane, (0, 0, 0), k))
    ph = np.linalg.solve(Ah, qo.incident_with_image(mesh, k, d, plane))
    rev = np.array([2, 1, 0, 5, 4, 3, 8, 7, 6])
    N2 = np.concatenate([nodes, plane.mirror(nodes)])
    E2 = np.concatenate([el, el[:, rev] + len(nodes)])
    m2 = qo.OrderMesh(N2, E2, order)
    e1, e2 = np.exp(1j * k * (m2.points @ d)), np.exp(1j * k * (plane.mirror(m2.points) @ d))
    b2 = e1 + e2 + bem.coupling(k) * 1j * k * ((m2.normals @ d) * e1 + (plane.reflect(m2.normals) @ d) * e2)
    p2 = np.linalg.solve(qo.dense_matrix(N2, E2, order, k), b2)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-0.6, 0.6, (10, 3))
    pts[:, 2] = rng.uniform(-0.25, 0.6, 10)
    pts = pts[np.linalg.norm(pts, axis=1) > 0.23]
    fh = qo.field_points_halfspace(nodes, el, order, np.eye(3), (1, 1, 1), k, ph, pts, d, plane)
    f2 = qo.field_points(N2, E2, order, np.eye(3), (1, 1, 1), k, p2, pts, d) + np.exp(1j * k * (plane.mirror(pts) @ d))
    assert np.abs(fh - f2).max() <= 1e-9 * np.abs(f2).max()


@pytest.mark.parametrize("order,counts", [(1, (4, 1, 1)), (2, (1, 1, 4))])
def test_fmm_image_product_tends_to_the_exact_image_part(order, counts):
    # the image part of the FMPBEM with V^ = R_p P2M of the reflected cell
    # (sign change on its double-layer term) converges to the exact image
    # blocks' product; a perpendicular axis (1, 1, 4) exercises the Hankel
    # part; without the sign change the product stalls near 0.2
    from oracle import halfspace
    from workloads import random_complex_vectors
    nodes, el = quad9_sphere(1, 0.2)
    plane = halfspace.Plane(2, -0.3, 0.8 - 0.3j)
    cell = qo.OrderMesh(nodes, el, order)
    L = np.eye(3)
    image = {d: qo.image_block(cell, L, counts, plane, d, 2.0, 0.3j) for d in bem.all_offsets(counts)}
    x = random_complex_vectors(9, 1, cell.n * cell.nb * 4)
    exact = bem.toeplitz_matvec(image, counts, halfspace.reverse_cells(x, counts, halfspace.hankel_axis(L, counts, plane)))
    errs = [np.linalg.norm(qo.fmm_image_matvec_explicit(cell, L, counts, 2.0, nt, plane, x, 0.3j) - exact)
            / np.linalg.norm(exact) for nt in (4, 8, 12)]
    assert errs[1] < 1e-3 * errs[0] and errs[2] < 1e-12, errs


def test_fmm2_near_block_with_higher_order_pressure():
    # the multilevel near field with shape-weighted leaf P2M tables and leaf
    # L2P tables at the nodes: order 0 through this path is the constant
    # element's; order 1 converges to the exact block (a leaf P2M that
    # spreads each element's moment evenly over its shapes stalls at 5e-4)
    from oracle import quad9 as q9
    L = np.diag([0.6, 0.6, 1.0])
    nodes, el = quad9_sphere(3, 0.2)
    A0 = qo.fmm2_near_block(qo.OrderMesh(nodes, el, 0), L, (0, 0, 0), 3.0, 6, 3, 0.3j)
    Aq = q9.fmm2_near_block(q9.Q9Mesh(nodes, el), L, (0, 0, 0), 3.0, 6, 3, 0.3j)
    assert np.abs(A0 - Aq).max() <= 1e-14 * np.abs(Aq).max()
    mesh = qo.OrderMesh(nodes, el, 1)
    S = qo.toeplitz_block(mesh, L, (0, 0, 0), 3.0, 0.3j)
    errs = [np.linalg.norm(qo.fmm2_near_block(mesh, L, (0, 0, 0), 3.0, ntn, 3, 0.3j) - S) / np.linalg.norm(S)
            for ntn in (4, 8)]
    assert errs[1] < 0.02 * errs[0] and errs[1] < 1e-6, errs

"""Pins of the oracle's half-space operator (Sec. 2.3, Sec. 3.4, Eq. (green3dHalf)):

* the image identity: a scatterer above a rigid (R_p = 1) or soft (R_p = -1)
  plane is the same problem as the scatterer and its mirror image in free
  space under the symmetric (antisymmetric) incident field, solved here with
  the full-space dense matrix of the doubled mesh (pinned by the analytic
  sphere series); the two solutions agree to the difference of the collapsed
  rules' apex on the mirrored elements (about 1e-9) and an error in the image
  geometry, its normals, a jump term or the reflected incident wave shows at
  O(1);
* the incident field with its image satisfies the plane's condition
  (dp/dn = 0 for R_p = 1 by central differences, p = 0 for R_p = -1), and its
  normal derivative matches central differences off the plane;
* R_p = 0 gives the full-space operator;
* the structured product (T + T^ P)(p) of Sec. 2.4 equals the dense
  half-space matrix assembled pair by pair, for a lattice parallel to the
  plane and for one with an axis perpendicular to it (the block Hankel case of
  Eq. (blockToeplizMatrixSymmetry)), and the dense image matrix is constant
  along the anti-diagonals of the perpendicular axis;
* the FMM image part S^ + U K^ V^ converges to the exact image product as
  n_t grows.
"""
import numpy as np
import pytest

from oracle import bem, halfspace as hs
from workloads import icosphere


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("Rp,kind,vec", [(1.0, "plane", [0.6, 0.0, -0.8]), (-1.0, "plane", [0.0, 0.6, -0.8]),
                                         (1.0, "monopole", [0.7, -0.2, 0.5])])
def test_image_identity_against_doubled_free_space_problem(Rp, kind, vec):
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    k = 3.0
    pl = hs.Plane(2, -0.3, Rp)
    A = hs.dense_matrix_halfspace(v, t, np.eye(3), (1, 1, 1), k, pl)
    p = np.linalg.solve(A, hs.rhs(cell, np.eye(3), (1, 1, 1), k, kind, vec, 1.0, pl))
    V2 = np.vstack([v, pl.mirror(v)])
    T2 = np.vstack([t, hs.image_tris(t) + len(v)])
    m2 = bem.CellMesh(V2, T2)
    A2 = bem.dense_matrix(V2, T2, np.eye(3), (1, 1, 1), k)
    pin, dpin = hs.incident(m2.centroid, m2.normal, k, kind, vec, 1.0, pl)
    p2 = np.linalg.solve(A2, pin + bem.coupling(k) * dpin)
    n = len(t)
    assert _rel(p2[:n], p) < 1e-8
    assert _rel(p2[n:], Rp * p) < 1e-7
    # the plane matters: the free-space solution is far from it
    pfree = np.linalg.solve(bem.dense_matrix(v, t, np.eye(3), (1, 1, 1), k),
                            hs.rhs(cell, np.eye(3), (1, 1, 1), k, kind, vec, 1.0))
    assert _rel(pfree, p) > 0.05


@pytest.mark.parametrize("kind,vec", [("plane", [0.48, 0.6, -0.64]), ("monopole", [0.3, -0.4, 0.9])])
def test_incident_field_satisfies_the_plane_condition(kind, vec):
    rng = np.random.default_rng(5)
    k, off = 4.0, -0.25
    pts = rng.uniform(-1, 1, size=(6, 3))
    pts[:, 2] = off
    ez = np.zeros_like(pts) + np.array([0.0, 0.0, 1.0])
    h = 1e-5
    hard = hs.Plane(2, off, 1.0)
    up, _ = hs.incident(pts + h * ez, ez, k, kind, vec, 1.0, hard)
    dn, _ = hs.incident(pts - h * ez, ez, k, kind, vec, 1.0, hard)
    pc, _ = hs.incident(pts, ez, k, kind, vec, 1.0, hard)
    assert np.abs((up - dn) / (2 * h)).max() < 1e-8 * np.abs(pc).max() * k
    soft = hs.Plane(2, off, -1.0)
    ps, _ = hs.incident(pts, ez, k, kind, vec, 1.0, soft)
    assert np.abs(ps).max() < 1e-14
    # dp/dn off the plane against central differences along random normals
    x = rng.uniform(-1, 1, size=(6, 3)) + np.array([0, 0, 0.5])
    nrm = rng.normal(size=(6, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    _, dp = hs.incident(x, nrm, k, kind, vec, 0.7 - 0.2j, hard)
    a, _ = hs.incident(x + h * nrm, nrm, k, kind, vec, 0.7 - 0.2j, hard)
    b, _ = hs.incident(x - h * nrm, nrm, k, kind, vec, 0.7 - 0.2j, hard)
    assert np.abs((a - b) / (2 * h) - dp).max() < 1e-6 * np.abs(dp).max()


def test_zero_reflection_is_the_full_space_operator():
    v, t = icosphere(0, 0.2)
    cell = bem.CellMesh(v, t)
    counts, L, k = (3, 2, 1), np.diag([0.5, 0.5, 1.0]), 2.5
    x = np.random.default_rng(1).normal(size=(2, cell.n * 6)) + 0j
    y0 = hs.structured_matvec_halfspace(cell, L, counts, k, hs.Plane(2, -0.3, 0.0), x)
    blocks = {d: bem.toeplitz_block(cell, L, d, k) for d in bem.all_offsets(counts)}
    assert np.array_equal(y0, bem.toeplitz_matvec(blocks, counts, x))


CASES = {
    # lattice parallel to the plane z = -0.3 (translation invariant G_h)
    "parallel": ((3, 2, 1), np.diag([0.5, 0.5, 1.0]), hs.Plane(2, -0.3, 1.0), -1),
    # cells stacked along z, perpendicular to the plane: block Hankel image part
    "perpendicular": ((2, 1, 3), np.diag([0.5, 1.0, 0.55]), hs.Plane(2, -0.26, 0.8 - 0.3j), 2),
    # a perpendicular x axis and a parallel y axis, soft plane x = 0.27
    "perpendicular_x": ((3, 2, 1), np.diag([-0.5, 0.45, 1.0]), hs.Plane(0, 0.27, -1.0), 0),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("beta", [0.0, 0.4 + 0.3j])
def test_structured_product_equals_dense_halfspace_matrix(case, beta):
    counts, L, pl, h = CASES[case]
    v, t = icosphere(0, 0.2)
    cell = bem.CellMesh(v, t)
    k = 3.5
    assert hs.hankel_axis(L, counts, pl) == h
    A = hs.dense_matrix_halfspace(v, t, L, counts, k, pl, beta)
    x = np.random.default_rng(2).normal(size=(2, A.shape[0])) + 1j * np.random.default_rng(3).normal(size=(2, A.shape[0]))
    y = hs.structured_matvec_halfspace(cell, L, counts, k, pl, x, beta)
    assert _rel(y, x @ A.T) < 1e-12


def test_image_matrix_is_block_hankel_along_the_perpendicular_axis():
    counts, L, pl, h = CASES["perpendicular"]
    v, t = icosphere(0, 0.2)
    k = 3.5
    Ah = (hs.dense_matrix_halfspace(v, t, L, counts, k, pl) - bem.dense_matrix(v, t, L, counts, k))
    n = len(t)
    cells = bem.lattice_cells(counts)
    blk = lambda a, b: Ah[a * n:(a + 1) * n, b * n:(b + 1) * n]
    for a, ca in enumerate(cells):
        for b, cb in enumerate(cells):
            for a2, ca2 in enumerate(cells):
                for b2, cb2 in enumerate(cells):
                    same = (ca[0] - cb[0] == ca2[0] - cb2[0] and ca[1] - cb[1] == ca2[1] - cb2[1]
                            and ca[2] + cb[2] == ca2[2] + cb2[2])
                    if same and (a, b) < (a2, b2):
                        assert np.abs(blk(a, b) - blk(a2, b2)).max() <= 1e-13 * np.abs(blk(a, b)).max()


def test_fmm_image_part_converges_to_the_exact_image_product():
    # spheres of radius 0.2 in cells of 0.7, stacked along z above a plane
    # 0.45 below the first centre: mirrored cells beyond 2 r are expanded
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    counts, L, pl = (3, 1, 4), np.diag([0.7, 1.0, 0.7]), hs.Plane(2, -0.45, 0.9 + 0.2j)
    k = 2.0
    x = np.random.default_rng(4).normal(size=(1, cell.n * 12)) + 0j
    near = hs.image_near_offsets(L, counts, pl)
    assert 0 < len(near) < len(hs.image_offsets(counts))
    img = {d: hs.image_block(cell, L, counts, pl, d, k) for d in hs.image_offsets(counts)}
    exact = bem.toeplitz_matvec(img, counts, hs.reverse_cells(x, counts, 2))
    errs = [_rel(hs.fmm_image_matvec_explicit(cell, L, counts, k, nt, pl, x), exact) for nt in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5, errs

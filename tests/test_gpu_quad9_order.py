"""Parity of the CUDA paths on nine-node quadrilaterals that go beyond the
constant-pressure PBEM and FMM forms, through the C ABI, against the oracle:

* discontinuous pressure of order 1 (2 x 2 nodes) and 2 (eight-node
  serendipity), Sec. 2.1 Eq. (matrixBEM): blocks T_delta, PBEM products and
  solves against the dense matrix of the array, FP32 and MIXED products;
* the FMM form with pressure of order 1 and 2 (Eq. (2dPeriodicFMM), the P2M
  table weighted by the shapes, App. A Eq. (p2m));
* field points and the insertion loss (Eq. (cbie) with c = 1,
  Eq. (insertionloss)) for every order;
* the half-space Green's function (Sec. 2.3 Eq. (green3dHalf), Sec. 3.4
  Eq. (2dPeriodicFMM_halfspace)) in the PBEM and FMM forms, with and without
  an axis perpendicular to the plane (block Hankel image part);
* the FMPBEM2 form (Sec. 3.3) on constant-pressure quadrilateral cells.

Tolerances (relative to the largest entry of a block, or relative L2 for
products).  Regular entries 1e-12: the same FP64 rules on both sides.  Self
entries 5e-9: the oracle forms y - x about an off-centre node from absolute
node coordinates, and the finite-part subtraction amplifies that rounding by
(rho_hat / rho_min)^2, up to 4e6 on the thin triangles towards the nearest
side; the CUDA path forms y - x from the element's monomials about the node.
Products and solutions that include self entries: 5e-9.  Field points use
only regular rules: 1e-12.  FMPBEM2 on constant pressure: 1e-10 (its exact
entries include the centre-node self terms, 1e-10 in the constant-pressure
tests).  FP32 operators: 1e-5 against the FP64 product.
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm, halfspace as hs, quad9, quad9_order as qo
from workloads import quad9_sphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

LATTICE = np.diag([0.5, 0.55, 1.0])
NB = {0: 1, 1: 4, 2: 8}


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _array(nodes, el, counts, L):
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, float) @ L for c in cells])
    allE = np.concatenate([el + i * len(nodes) for i in range(len(cells))])
    return allN, allE


def _fluid_points(centres, n, rmin, rmax, seed):
    """n points at distances rmin..rmax from the given sphere centres and
    farther than rmin from every centre."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        c = centres[rng.integers(len(centres))]
        d = rng.normal(size=3)
        x = c + rng.uniform(rmin, rmax) * d / np.linalg.norm(d)
        if np.min(np.linalg.norm(centres - x, axis=1)) > rmin:
            out.append(x)
    return np.array(out)


# ----------------------------------------------------------- blocks ------

@pytest.mark.parametrize("order,m,counts,k,beta", [
    (1, 2, (3, 2, 1), 3.0, 0.0),            # 96 dofs per cell, every class, 15 offsets
    (2, 1, (3, 2, 1), 3.0, 0.3 + 0.2j),     # 48 dofs per cell, with an admittance
    (1, 1, (1, 1, 2), 9.0, 0.5 - 0.4j),     # 24 dofs per cell: a ragged tail of every warp
    (2, 2, (2, 1, 1), 5.0, 0.0),            # 192 dofs per cell
])
def test_q9p_blocks_match_oracle(order, m, counts, k, beta):
    nodes, el = quad9_sphere(m, 0.2)
    lat = LATTICE if counts[2] == 1 else np.diag([1.0, 1.0, 0.45])
    offs = bem.all_offsets(counts)
    T = gb.build_blocks_q9(nodes, el, counts, lat, k, offs, beta=beta, pressure_order=order).cpu().numpy()
    cell = qo.OrderMesh(nodes, el, order)
    nd = cell.n * cell.nb
    assert T.shape == (len(offs), nd, nd)
    same_elem = np.kron(np.eye(cell.n, dtype=bool), np.ones((cell.nb, cell.nb), dtype=bool))
    for o, d in enumerate(offs):
        ref = qo.toeplitz_block(cell, lat, d, k, beta)
        scale = np.abs(ref).max()
        reg = ~same_elem if not np.any(d) else np.ones_like(same_elem)
        assert np.abs(T[o] - ref)[reg].max() <= 1e-12 * scale, d
        if not np.any(d):
            assert np.abs(T[o] - ref)[same_elem].max() <= 5e-9 * scale


# ------------------------------------------------------ PBEM products ----

@pytest.mark.parametrize("order", [1, 2])
def test_q9p_operator_matvec_and_solve_match_dense_oracle(order):
    nodes, el = quad9_sphere(1, 0.2)
    counts, k = (2, 2, 1), 3.0
    op = gb.Operator(nodes, el, counts, LATTICE, k, pressure_order=order)
    assert op.info["pressure_order"] == order and op.info["form_name"] == "pbem"
    assert op.info["n"] == len(el) * NB[order]
    allN, allE = _array(nodes, el, counts, LATTICE)
    A = qo.dense_matrix(allN, allE, order, k)
    x = random_complex_vectors(61, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    assert _rel(y, x @ A.T) < 5e-9
    d = [0.6, 0.8, 0.0]
    b = op.rhs_plane_wave([d])
    bref = qo.plane_wave_rhs(qo.OrderMesh(allN, allE, order), k, d)
    assert _rel(b.cpu().numpy()[0], bref) < 1e-13
    p, info = op.solve(b, tol=1e-11)
    assert info[0]["converged"]
    assert _rel(p.cpu().numpy()[0], np.linalg.solve(A, bref)) < 5e-8


@pytest.mark.parametrize("order", [1, 2])
def test_q9p_reduced_precision_products(order):
    nodes, el = quad9_sphere(1, 0.2)
    counts, k = (3, 2, 1), 4.0
    x = _dev(random_complex_vectors(62, 1, len(el) * NB[order] * 6))
    y64 = gb.Operator(nodes, el, counts, LATTICE, k, pressure_order=order).matvec(x)
    for prec in (gb.FP32, gb.MIXED):
        yp = gb.Operator(nodes, el, counts, LATTICE, k, precision=prec, pressure_order=order).matvec(x)
        assert float(torch.linalg.vector_norm(yp - y64) / torch.linalg.vector_norm(y64)) < 1e-5, prec


def test_q9p_mixed_solve_reaches_the_fp64_solution():
    nodes, el = quad9_sphere(1, 0.2)
    counts, k = (3, 2, 1), 3.0
    sols = []
    for prec in (gb.FP64, gb.MIXED):
        op = gb.Operator(nodes, el, counts, LATTICE, k, precision=prec, pressure_order=2)
        p, info = op.solve(op.rhs_plane_wave([[1.0, 0.0, 0.0]]), tol=1e-10)
        assert info[0]["converged"]
        sols.append(p)
    assert float(torch.linalg.vector_norm(sols[1] - sols[0]) / torch.linalg.vector_norm(sols[0])) < 1e-8


# ------------------------------------------------------- FMM form --------

@pytest.mark.parametrize("order,beta", [(1, 0.0), (2, 0.3 + 0.2j)])
def test_q9p_fmm_matvec_equals_explicit_oracle(order, beta):
    nodes, el = quad9_sphere(1, 0.2)
    L, counts, k, nt = np.eye(3), (4, 1, 1), 2.0, 6
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta, pressure_order=order)
    assert op.info["form_name"] == "fmm" and op.info["pressure_order"] == order
    x = random_complex_vectors(63, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = qo.fmm_matvec_explicit(qo.OrderMesh(nodes, el, order), L, counts, k, nt, x, beta)
    assert _rel(y, ref) < 5e-9
    op32 = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta, precision=gb.FP32,
                       pressure_order=order)
    assert _rel(op32.matvec(_dev(x)).cpu().numpy(), y) < 1e-5


def test_q9p_fmm_solve_tends_to_the_pbem_solve():
    nodes, el = quad9_sphere(1, 0.2)
    L, counts, k = np.eye(3), (5, 2, 1), 2.0
    sols = {}
    for name, form, nt in (("pbem", gb.FORM_PBEM, 0), ("fmm", gb.FORM_FMM, 10)):
        op = gb.Operator(nodes, el, counts, L, k, form=form, n_t=nt, pressure_order=1)
        p, info = op.solve(op.rhs_plane_wave([[1.0, 0.0, 0.0]]), tol=1e-11)
        assert info[0]["converged"]
        sols[name] = p
    assert float(torch.linalg.vector_norm(sols["fmm"] - sols["pbem"]) / torch.linalg.vector_norm(sols["pbem"])) < 1e-8


# ------------------------------------------- field points, insertion loss --

@pytest.mark.parametrize("order,m,beta", [(0, 2, 0.0), (1, 1, 0.3 + 0.2j), (2, 1, 0.0)])
def test_q9_field_points_match_oracle(order, m, beta):
    nodes, el = quad9_sphere(m, 0.2)
    counts, k = (2, 1, 1), 3.0
    op = gb.Operator(nodes, el, counts, LATTICE, k, beta=beta, pressure_order=order)
    p = random_complex_vectors(64, 2, op.N)
    centres = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    # very near (0.21), near and far points of both spheres
    pts = np.vstack([_fluid_points(centres, 6, 0.21, 0.24, 5), _fluid_points(centres, 6, 0.25, 0.9, 6)])
    dirs = [[1.0, 0.0, 0.0], [0.0, 0.6, 0.8]]
    out = op.field(_dev(p), dirs, pts, amps=[1.0, 0.5 - 0.25j]).cpu().numpy()
    for r, amp in enumerate((1.0, 0.5 - 0.25j)):
        ref = qo.field_points(nodes, el, order, LATTICE, counts, k, p[r], pts, dirs[r], amp=amp, beta=beta)
        assert _rel(out[r], ref) < 1e-12, r


@pytest.mark.parametrize("order", [0, 2])
def test_q9_insertion_loss_matches_oracle(order):
    nodes, el = quad9_sphere(1, 0.2)
    counts, k = (2, 1, 1), 3.0
    op = gb.Operator(nodes, el, counts, LATTICE, k, pressure_order=order)
    incs = [("plane", [1.0, 0.0, 0.0], 1.0), ("plane", [0.0, 0.6, 0.8], 0.5 - 0.25j)]
    b = op.rhs_incident(incs)
    p, info = op.solve(b, tol=1e-10)
    assert all(i["converged"] for i in info)
    pts = np.stack(np.meshgrid(np.linspace(1.0, 1.6, 5), np.linspace(-0.4, 0.4, 4), [0.3]), -1).reshape(-1, 3)
    il = op.insertion_loss(p, incs, pts)
    P = p.cpu().numpy()
    tot = sum(qo.field_points(nodes, el, order, LATTICE, counts, k, P[r], pts, v, amp=a) for r, (_, v, a) in
              enumerate(incs))
    inc = sum(a * np.exp(1j * k * (pts @ np.asarray(v))) for _, v, a in incs)
    ref = hs.insertion_loss_from_fields(inc, tot)
    assert abs(il - ref) < 1e-9, (il, ref)


# --------------------------------------------------------- half-space ----

HS_CASES = {
    "parallel": ((3, 2, 1), np.diag([0.5, 0.45, 1.0]), (2, -0.3, 1.0), -1),
    "perpendicular": ((2, 1, 2), np.diag([0.5, 1.0, 0.45]), (2, -0.3, 0.8 - 0.3j), 2),
}


@pytest.mark.parametrize("case", list(HS_CASES))
@pytest.mark.parametrize("order,beta", [(0, 0.0), (1, 0.3 + 0.2j), (2, 0.0)])
def test_q9_halfspace_pbem_matvec_equals_dense_oracle(case, order, beta):
    counts, L, plane, h = HS_CASES[case]
    nodes, el = quad9_sphere(1, 0.2)
    k = 3.0
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_PBEM, beta=beta, plane=plane, pressure_order=order)
    assert op.info["halfspace"] == 1 and op.info["hankel_axis"] == h
    x = random_complex_vectors(65, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    A = qo.dense_matrix_halfspace(nodes, el, order, L, counts, k, hs.Plane(*plane), beta)
    assert _rel(y, x @ A.T) < 5e-9
    if order == 1:
        op32 = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_PBEM, beta=beta, plane=plane, pressure_order=order,
                           precision=gb.FP32)
        assert _rel(op32.matvec(_dev(x)).cpu().numpy(), y) < 1e-5


@pytest.mark.parametrize("order", [0, 2])
def test_q9_halfspace_rhs_field_and_solve_match_oracle(order):
    counts, L, plane, h = HS_CASES["perpendicular"]
    nodes, el = quad9_sphere(1, 0.2)
    k, d = 3.0, [0.6, 0.0, -0.8]
    pl = hs.Plane(*plane)
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_PBEM, plane=plane, pressure_order=order)
    allN, allE = _array(nodes, el, counts, L)
    b = op.rhs_plane_wave([d])
    bref = qo.incident_with_image(qo.OrderMesh(allN, allE, order), k, d, pl)
    assert _rel(b.cpu().numpy()[0], bref) < 1e-13
    p, info = op.solve(b, tol=1e-11, restart=60)
    assert info[0]["converged"]
    A = qo.dense_matrix_halfspace(nodes, el, order, L, counts, k, pl)
    pref = np.linalg.solve(A, bref)
    assert _rel(p.cpu().numpy()[0], pref) < 5e-8
    centres = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.45], [0.5, 0.0, 0.45]])
    pts = _fluid_points(centres, 10, 0.21, 0.5, 7)
    pts = pts[pts[:, 2] > -0.25]
    out = op.field(p, [d], pts).cpu().numpy()[0]
    ref = qo.field_points_halfspace(nodes, el, order, L, counts, k, p.cpu().numpy()[0], pts, d, pl)
    assert _rel(out, ref) < 1e-12


@pytest.mark.parametrize("order,precision,tol", [(0, "FP64", 5e-9), (1, "FP64", 5e-9), (2, "FP32", 1e-5)])
def test_q9_halfspace_fmm_matvec_equals_explicit_oracle(order, precision, tol):
    counts, L, plane = (3, 1, 4), np.diag([0.7, 1.0, 0.7]), (2, -0.45, 0.9 + 0.2j)
    nodes, el = quad9_sphere(1, 0.2)
    k, nt = 2.0, 6
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, precision=getattr(gb, precision),
                     plane=plane, pressure_order=order)
    pl = hs.Plane(*plane)
    assert op.info["form_name"] == "fmm" and op.info["n_near_image"] == len(hs.image_near_offsets(L, counts, pl))
    x = random_complex_vectors(66, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    cell = qo.OrderMesh(nodes, el, order)
    ref = qo.fmm_matvec_explicit(cell, L, counts, k, nt, x) + qo.fmm_image_matvec_explicit(cell, L, counts, k, nt,
                                                                                           pl, x)
    assert _rel(y, ref) < tol


def test_q9_halfspace_fmm_parallel_lattice_with_admittance():
    nodes, el = quad9_sphere(1, 0.2)
    counts, L, plane, k, nt, beta = (4, 3, 1), np.diag([0.7, 0.7, 1.0]), (2, -0.5, -1.0), 2.5, 6, 0.3 + 0.2j
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta, plane=plane, pressure_order=1)
    assert op.info["hankel_axis"] == -1 and op.info["image_separate"] == 1
    x = random_complex_vectors(67, 1, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    cell = qo.OrderMesh(nodes, el, 1)
    pl = hs.Plane(*plane)
    ref = (qo.fmm_matvec_explicit(cell, L, counts, k, nt, x, beta)
           + qo.fmm_image_matvec_explicit(cell, L, counts, k, nt, pl, x, beta))
    assert _rel(y, ref) < 5e-9


# ------------------------------------------------------------ FMPBEM2 ----

@pytest.mark.parametrize("levels,ntn,beta", [(1, 4, 0.0), (2, 6, 0.0), (2, 5, 0.3 + 0.2j)])
def test_q9_fmm2_matvec_equals_explicit_oracle(levels, ntn, beta):
    nodes, el = quad9_sphere(2, 0.2)
    counts, L, k, nt = (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 3.0, 6
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM2, n_t=nt, n_t_near=ntn, near_levels=levels, beta=beta)
    assert op.info["form_name"] == "fmm2" and op.info["element"] == gb.ELEM_QUAD9
    assert op.info["near_levels"] == levels
    x = random_complex_vectors(68, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = quad9.fmm2_matvec_explicit(quad9.Q9Mesh(nodes, el), L, counts, k, nt, ntn, levels, x, beta)
    assert _rel(y, ref) < 1e-10


def test_q9_fmm2_converges_to_the_fmm_form():
    nodes, el = quad9_sphere(3, 0.2)
    counts, L, k = (4, 3, 1), np.diag([0.6, 0.6, 1.0]), 3.0
    x = _dev(random_complex_vectors(69, 1, len(el) * 12))
    y_fmm = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=6).matvec(x)
    errs = []
    for ntn in (3, 6, 9):
        op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM2, n_t=6, n_t_near=ntn, near_levels=2)
        errs.append(float(torch.linalg.vector_norm(op.matvec(x) - y_fmm) / torch.linalg.vector_norm(y_fmm)))
    # each step of 3 in n_t,near cuts the distance at least four-fold (the
    # curved cell's leaf boxes are measured over all nine nodes, so the
    # ratio is slower than on the flat triangles' cell)
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4 and errs[2] < 2e-4, errs

"""Parity of the CUDA path on nine-node quadratic quadrilaterals (Sec. 2.1,
Eq. (matrixBEM); constant pressure collocated at the element centre) with the
oracle, through the C ABI.

Tolerances.  Regular entries: 1e-12 of the block's largest entry (the same
rules in FP64 on both sides).  Self entries: 1e-10 of it.  The oracle forms
y - x near the collocation point from absolute node coordinates, and the
finite-part subtraction F - F_-2/rho^2 - F_-1/rho multiplies that rounding
by (rho_hat / rho_min)^2 (about 4e4 for the 16-point rule).  The CUDA path
forms y - x from the element's monomial coefficients about the centre.  The
two agree to about 2e-11 of the entry.  Operator products and solutions
carry the same bound.
"""
import numpy as np
import pytest
import torch
from scipy.special import eval_legendre

from oracle import bem, quad9
from oracle.special import sph_hn_deriv
from workloads import quad9_sphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

LATTICE = np.diag([0.5, 0.55, 1.0])


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _array(nodes, el, counts):
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, float) @ LATTICE for c in cells])
    allE = np.concatenate([el + i * len(nodes) for i in range(len(cells))])
    return allN, allE


@pytest.mark.parametrize("m,counts,k,beta", [
    (3, (3, 2, 1), 3.0, 0.0),           # 54 elements: every class, 15 offsets
    (3, (3, 2, 1), 3.0, 0.3 + 0.2j),    # with an admittance (S and K terms)
    (1, (2, 1, 1), 7.0, 0.0),           # 6 elements: a ragged tail of every warp
    (2, (1, 1, 2), 11.0, 0.5 - 0.4j),   # 24 elements stacked along z
])
def test_q9_blocks_match_oracle(m, counts, k, beta):
    nodes, el = quad9_sphere(m, 0.2)
    lat = LATTICE if counts[2] == 1 else np.diag([1.0, 1.0, 0.45])
    offs = bem.all_offsets(counts)
    T = gb.build_blocks_q9(nodes, el, counts, lat, k, offs, beta=beta).cpu().numpy()
    cell = quad9.Q9Mesh(nodes, el)
    for o, d in enumerate(offs):
        ref = quad9.toeplitz_block(cell, lat, d, k, beta)
        scale = np.abs(ref).max()
        off = ~np.eye(cell.n, dtype=bool) if not np.any(d) else np.ones_like(ref, dtype=bool)
        assert np.abs(T[o] - ref)[off].max() <= 1e-12 * scale, d
        if not np.any(d):
            assert np.abs(np.diag(T[o]) - np.diag(ref)).max() <= 1e-10 * scale


def test_q9_operator_matvec_and_solve_match_dense_oracle():
    nodes, el = quad9_sphere(2, 0.2)
    counts, k = (2, 2, 1), 3.0
    op = gb.Operator(nodes, el, counts, LATTICE, k)
    assert op.info["element"] == gb.ELEM_QUAD9 and op.info["form_name"] == "pbem" and op.info["n"] == 24
    allN, allE = _array(nodes, el, counts)
    A = quad9.dense_matrix(allN, allE, k)
    x = random_complex_vectors(51, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    assert _rel(y, x @ A.T) < 1e-10
    d = [0.6, 0.8, 0.0]
    b = op.rhs_plane_wave([d])
    bref = quad9.plane_wave_rhs(quad9.Q9Mesh(allN, allE), k, d)
    assert _rel(b.cpu().numpy()[0], bref) < 1e-13
    p, info = op.solve(b, tol=1e-11)
    assert info[0]["converged"]
    assert _rel(p.cpu().numpy()[0], np.linalg.solve(A, bref)) < 1e-9


def test_q9_reduced_precision_products():
    nodes, el = quad9_sphere(2, 0.2)
    counts, k = (3, 2, 1), 4.0
    x = _dev(random_complex_vectors(52, 1, 24 * 6))
    y64 = gb.Operator(nodes, el, counts, LATTICE, k).matvec(x)
    for prec in (gb.FP32, gb.MIXED):
        op = gb.Operator(nodes, el, counts, LATTICE, k, precision=prec)
        yp = op.matvec(x)
        assert float(torch.linalg.vector_norm(yp - y64) / torch.linalg.vector_norm(y64)) < 1e-5, prec


@pytest.mark.parametrize("beta", [0.0, 0.3 + 0.2j])
def test_q9_fmm_matvec_equals_explicit_oracle(beta):
    # FMPBEM on the curved elements: near blocks from the Q9 quadrature, the
    # P2M table over the 4 x 4 far rule with each point's normal
    nodes, el = quad9_sphere(2, 0.2)
    L, counts, k, nt = np.eye(3), (4, 1, 1), 2.0, 6
    op = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta)
    assert op.info["form_name"] == "fmm" and op.info["element"] == gb.ELEM_QUAD9
    x = random_complex_vectors(53, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = quad9.fmm_matvec_explicit(quad9.Q9Mesh(nodes, el), L, counts, k, nt, x, beta)
    assert _rel(y, ref) < 1e-10
    op32 = gb.Operator(nodes, el, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta, precision=gb.FP32)
    assert _rel(op32.matvec(_dev(x)).cpu().numpy(), y) < 1e-5


def test_q9_fmm_solve_tends_to_the_pbem_solve():
    nodes, el = quad9_sphere(2, 0.2)
    L, counts, k = np.eye(3), (5, 2, 1), 2.0
    sols = {}
    for name, form, nt in (("pbem", gb.FORM_PBEM, 0), ("fmm", gb.FORM_FMM, 10)):
        op = gb.Operator(nodes, el, counts, L, k, form=form, n_t=nt)
        b = op.rhs_plane_wave([[1.0, 0.0, 0.0]])
        p, info = op.solve(b, tol=1e-11)
        assert info[0]["converged"]
        sols[name] = p
    assert float(torch.linalg.vector_norm(sols["fmm"] - sols["pbem"]) / torch.linalg.vector_norm(sols["pbem"])) < 1e-9


def _series(ka, ct, nmax=40):
    return sum((2 * n + 1) * 1j ** n * (1j / ka ** 2) / sph_hn_deriv(n, ka) * eval_legendre(n, ct)
               for n in range(nmax))


def test_q9_rigid_sphere_against_the_analytic_series():
    # an independent pin of the whole GPU path: the scattered sphere
    k, a = 2.0, 0.2
    errs = []
    for m in (2, 4):
        nodes, el = quad9_sphere(m, a)
        op = gb.Operator(nodes, el, (1, 1, 1), np.eye(3), k)
        p, info = op.solve(op.rhs_plane_wave([[1.0, 0.0, 0.0]]), tol=1e-10)
        assert info[0]["converged"]
        cen = quad9.Q9Mesh(nodes, el).centroid
        pa = _series(k * a, cen[:, 0] / np.linalg.norm(cen, axis=1))
        errs.append(_rel(p.cpu().numpy()[0], pa))
    assert errs[1] < 0.3 * errs[0] and errs[1] < 6e-3, errs


def test_q9_argument_errors():
    nodes, el = quad9_sphere(1, 0.2)
    counts = (2, 1, 1)
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, form=gb.FORM_FMM2, precision=gb.FP32)
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, form=gb.FORM_FMM, precision=gb.MIXED)
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, form=gb.FORM_FMM2, plane=(2, -0.3, 1.0))
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, precision=gb.BF16)
    bad = el.copy()
    bad[0, 4] = len(nodes)
    with pytest.raises(gb.FmpbError, match="EMESH"):
        gb.Operator(nodes, bad, counts, LATTICE, 2.0)
    flat = el.copy()
    flat[0, :] = flat[0, 0]      # all nine nodes on one point: no Jacobian
    with pytest.raises(gb.FmpbError, match="EMESH"):
        gb.build_blocks_q9(nodes, flat, counts, LATTICE, 2.0, [[0, 0, 0]])
    # refused before any device work: pressure of order 1, 2 with the
    # FMPBEM2 form, and an order that does not exist
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, form=gb.FORM_FMM2, pressure_order=1)
    with pytest.raises(gb.FmpbError):
        gb.Operator(nodes, el, counts, LATTICE, 2.0, pressure_order=3)

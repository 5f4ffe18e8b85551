"""Parity of the CUDA FMPBEM2 form (Sec. 3.3: near blocks as a multilevel FMM
over the unit cell's octree) with the oracle, through the C ABI.

Tolerances: 1e-12 relative against the oracle's explicit FMPBEM2 product
(FP64 arithmetic on both sides; the regular translations agree to 1e-13);
the FMPBEM2 product converges to the FMM form's as n_t,near grows; the
solved pressure within 1e-3 of the dense oracle.
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm2
from workloads import icosphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

COUNTS, LATTICE = (4, 3, 1), np.diag([0.6, 0.6, 1.0])


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("levels,ntn,beta", [(2, 6, 0.0), (1, 4, 0.0), (2, 5, 0.3 + 0.2j), (3, 6, 0.0)])
def test_fmm2_matvec_equals_explicit_oracle(levels, ntn, beta):
    v, t = icosphere(1, 0.2)
    k, nt = 3.0, 6
    op = gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM2, n_t=nt, n_t_near=ntn, near_levels=levels,
                     beta=beta)
    assert op.info["form_name"] == "fmm2" and op.info["near_levels"] == levels
    x = random_complex_vectors(41, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = fmm2.fmm2_matvec_explicit(bem.CellMesh(v, t), LATTICE, COUNTS, k, nt, ntn, levels, x, beta=beta)
    assert _rel(y, ref) < 1e-12


def test_fmm2_converges_to_the_fmm_form():
    v, t = icosphere(2, 0.2)
    k = 3.0
    x = _dev(random_complex_vectors(42, 1, 320 * 12))
    y_fmm = gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM, n_t=6).matvec(x)
    errs = []
    for ntn in (3, 6, 9):
        op = gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_FMM2, n_t=6, n_t_near=ntn, near_levels=2)
        errs.append(float(torch.linalg.vector_norm(op.matvec(x) - y_fmm) / torch.linalg.vector_norm(y_fmm)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4, errs


def test_fmm2_solve_matches_dense_oracle():
    v, t = icosphere(1, 0.2)
    counts, k = (3, 2, 1), 3.0
    op = gb.Operator(v, t, counts, LATTICE, k, form=gb.FORM_FMM2, n_t=8, n_t_near=8, near_levels=2)
    b = op.rhs_plane_wave([[0.6, 0.8, 0.0]])
    p, info = op.solve(b, tol=1e-10)
    A = bem.dense_matrix(v, t, LATTICE, counts, k)
    pref = np.linalg.solve(A, b.cpu().numpy()[0])
    assert info[0]["converged"]
    assert _rel(p.cpu().numpy()[0], pref) < 1e-3


def test_fmm2_argument_errors():
    v, t = icosphere(0, 0.2)
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM2, precision=gb.FP32)
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM2, near_levels=11)
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, COUNTS, LATTICE, 2.0, form=gb.FORM_FMM2, plane=(2, -0.3, 1.0))

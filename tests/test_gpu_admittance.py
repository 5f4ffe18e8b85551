"""Parity of the CUDA admittance path (Eq. (admittance) in Eq. (bm)) with the
oracle, through the C ABI, on seeded inputs.

Tolerances as for the rigid path: 1e-12 relative for blocks, tables and FP64
products; the solved pressure within 1e-3 of the dense oracle (the FMM
truncation error) and 1e-9 for the PBEM form (exact up to rounding).
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm
from workloads import WORKLOADS, icosphere, cube, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

BETAS = [0.5 + 0.3j, 1.0, 0.2 - 0.7j]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("mesh,counts,lattice,k,beta", [
    ("ico1", (2, 2, 1), np.diag([0.5, 0.45, 1.0]), 3.0, BETAS[0]),
    ("cube", (2, 1, 1), np.diag([0.5, 0.5, 0.5]), 6.0, BETAS[1]),
    ("ico1", (3, 1, 1), np.diag([0.41, 1.0, 1.0]), 11.0, BETAS[2]),
])
def test_admittance_blocks_match_oracle(mesh, counts, lattice, k, beta):
    # every offset of the grid: self, near, very-near and far classes
    v, t = {"ico1": lambda: icosphere(1, 0.2), "cube": lambda: cube(0.3, 4)}[mesh]()
    offs = bem.all_offsets(counts)
    T = gb.build_blocks_admittance(v, t, counts, lattice, k, beta, offs).cpu().numpy()
    cell = bem.CellMesh(v, t)
    for o, d in enumerate(offs):
        ref = bem.toeplitz_block(cell, lattice, d, k, beta)
        assert np.abs(T[o] - ref).max() <= 1e-12 * np.abs(ref).max(), d


def test_zero_admittance_is_the_rigid_build_bit_for_bit():
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (2, 2, 1), np.diag([0.5, 0.45, 1.0]), 3.0
    offs = bem.all_offsets(counts)
    a = gb.build_blocks(v, t, counts, lattice, k, offs)
    b = gb.build_blocks_admittance(v, t, counts, lattice, k, 0.0, offs)
    assert torch.equal(a, b)
    V0, U0 = gb.multipole_tables(v, t, k, 5)
    V1, U1 = gb.multipole_tables_admittance(v, t, k, 0.0, 5)
    assert torch.equal(V0, V1) and torch.equal(U0, U1)


def test_admittance_changes_only_the_single_layer_terms():
    # T(beta) - T(0) = beta (1/2 delta - i k (S + (i/k) K)): linear in beta
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 4.0
    offs = bem.all_offsets(counts)
    T0 = gb.build_blocks(v, t, counts, lattice, k, offs).cpu().numpy()
    T1 = gb.build_blocks_admittance(v, t, counts, lattice, k, 1.0, offs).cpu().numpy()
    Tb = gb.build_blocks_admittance(v, t, counts, lattice, k, 0.3 - 0.8j, offs).cpu().numpy()
    assert _rel(Tb - T0, (0.3 - 0.8j) * (T1 - T0)) < 1e-13


def test_admittance_p2m_table_matches_oracle():
    v, t = icosphere(1, 0.2)
    k, nt, beta = 2.5, 6, BETAS[0]
    V0, U0 = gb.multipole_tables_admittance(v, t, k, beta, nt)
    cell = bem.CellMesh(v, t)
    assert _rel(V0.cpu().numpy(), fmm.p2m_table(cell, k, nt, beta)) < 1e-12
    assert _rel(U0.cpu().numpy(), fmm.l2p_table(cell, k, nt)) < 1e-12


@pytest.mark.parametrize("precision,tol", [("FP64", 1e-12), ("FP32", 1e-5)])
def test_admittance_pbem_matvec_equals_dense_oracle(precision, tol):
    v, t = icosphere(1, 0.2)
    counts, lattice, k, beta = (3, 2, 1), np.diag([0.5, 0.6, 1.0]), 3.0, BETAS[0]
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, precision=getattr(gb, precision), beta=beta)
    assert complex(op.info["beta_re"], op.info["beta_im"]) == beta
    x = random_complex_vectors(21, 3, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    A = bem.dense_matrix(v, t, lattice, counts, k, beta)
    assert _rel(y, x @ A.T) < tol


@pytest.mark.parametrize("counts,lattice,k,nt,beta", [
    ((5, 1, 1), np.diag([0.6, 1.0, 1.0]), 2.0, 6, BETAS[1]),
    ((5, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0, 5, BETAS[2]),
])
def test_admittance_fmm_matvec_equals_explicit_oracle(counts, lattice, k, nt, beta):
    v, t = icosphere(1, 0.2)
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt, beta=beta)
    assert op.info["form_name"] == "fmm"
    x = random_complex_vectors(22, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = fmm.fmm_matvec_explicit(bem.CellMesh(v, t), lattice, counts, k, nt, x, beta=beta)
    assert _rel(y, ref) < 1e-12


def test_admittance_pbem_solve_matches_dense_oracle():
    v, t = icosphere(1, 0.2)
    counts, lattice, k, beta = (3, 3, 1), np.diag([0.45, 0.45, 1.0]), 5.0, BETAS[0]
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, beta=beta)
    b = op.rhs_plane_wave([[0.8, 0.6, 0.0]])
    p, info = op.solve(b, tol=1e-12, restart=40)
    A = bem.dense_matrix(v, t, lattice, counts, k, beta)
    pref = np.linalg.solve(A, b.cpu().numpy()[0])
    assert info[0]["converged"]
    assert _rel(p.cpu().numpy()[0], pref) < 1e-9


def test_admittance_fmm_solve_matches_dense_oracle():
    w = WORKLOADS["sphere_row_4"]
    v, t = w.mesh()
    k, beta = w.wavenumbers[0], BETAS[1]
    op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t, beta=beta)
    dirs = np.array([[1.0, 0, 0], [0.6, 0, -0.8]])
    b = op.rhs_plane_wave(dirs)
    p, info = op.solve(b, tol=1e-10)
    p = p.cpu().numpy()
    A = bem.dense_matrix(v, t, w.lattice, w.counts, k, beta)
    for r in range(2):
        pref = np.linalg.solve(A, b.cpu().numpy()[r])
        assert info[r]["converged"]
        assert _rel(p[r], pref) < 1e-3


def test_admittance_field_points_match_oracle():
    v, t = icosphere(1, 0.2)
    counts, lattice, k, beta = (2, 1, 1), np.diag([0.7, 1.0, 1.0]), 2.0, BETAS[2]
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, beta=beta)
    dirs = np.array([[1.0, 0, 0], [0, 0.6, 0.8]])
    amps = np.array([1.0, 0.5 - 0.25j])
    p = random_complex_vectors(23, 2, op.N)
    # far, near and very-near points (0.22 is within 1.5 h of the sphere)
    pts = np.array([[0.35, 0.1, 0.05], [-0.3, 0.2, 0.1], [0.35, 0.0, 0.45], [1.5, -0.5, 0.3], [0.22, 0.0, 0.0]])
    out = op.field(_dev(p), dirs, pts, amps).cpu().numpy()
    for r in range(2):
        ref = bem.field_points(v, t, lattice, counts, k, p[r], pts, dirs[r], amps[r], beta=beta)
        assert _rel(out[r], ref) < 1e-12


def test_admittance_is_refused_when_not_finite():
    v, t = icosphere(0, 0.2)
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 2.0, beta=complex(float("nan"), 0.0))
    with pytest.raises(gb.FmpbError):
        gb.build_blocks_admittance(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 2.0, float("inf"), [(0, 0, 0)])


class _Rows:
    def __init__(self, cell, rows):
        self.centroid = cell.centroid[rows]
        self.normal = cell.normal[rows]
        self.n = len(rows)


def test_admittance_sonic_crystal_full_size_sampled_rows():
    """3x20 capped cylinders, N = 72,000, PBEM form, beta = 0.4 + 0.2i:
    sampled rows of A x against the oracle's quadrature, row by row."""
    w = WORKLOADS["sonic_crystal_3x20"]
    v, t = w.mesh()
    k, beta = w.wavenumbers[2], 0.4 + 0.2j
    op = gb.Operator(v, t, w.counts, w.lattice, k, beta=beta)
    assert op.info["form_name"] == "pbem"
    x = random_complex_vectors(w.rhs_seed, 1, op.N)[0]
    y = op.matvec(_dev(x[None])).cpu().numpy()[0]
    cell = bem.CellMesh(v, t)
    n = cell.n
    cells = bem.lattice_cells(w.counts)
    L = np.asarray(w.lattice, dtype=float)
    for gi in [0, 35 * 1200 + 611, 59 * 1200 + 1187]:
        c, i = divmod(gi, n)
        acc = 0.0 + 0.0j
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(cells[c], cp))
            selfp = np.zeros((1, n), dtype=bool)
            if not any(delta):
                selfp[0, i] = True
            D, H, S, K = bem.dh_block(_Rows(cell, [i]), cell.v - np.asarray(delta, float) @ L, k,
                                      self_pairs=selfp, with_sk=True)
            row = bem._entries(D, H, S, K, k, beta)[0]
            if not any(delta):
                row[i] += 0.5 + 0.5 * beta
            acc += row @ x[cj * n:(cj + 1) * n]
        assert abs(y[gi] - acc) <= 1e-11 * abs(acc), gi

"""Parity of the CUDA half-space path (Sec. 2.3, Sec. 3.4, Eq. (green3dHalf))
with the oracle, through the C ABI.

Tolerances: 1e-12 relative for FP64 products, right-hand sides and field
points against the dense half-space matrix (or the oracle's explicit FMM
product), 1e-5 for FP32; solved pressure 1e-9 (PBEM form) and 1e-3 (FMM
truncation) against the dense solution.
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm, halfspace as hs
from workloads import WORKLOADS, icosphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


CASES = {
    "parallel": ((3, 2, 1), np.diag([0.5, 0.5, 1.0]), (2, -0.3, 1.0), -1),
    "perpendicular": ((2, 1, 3), np.diag([0.5, 1.0, 0.55]), (2, -0.26, 0.8 - 0.3j), 2),
    "perpendicular_x": ((3, 2, 1), np.diag([-0.5, 0.45, 1.0]), (0, 0.27, -1.0), 0),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("beta", [0.0, 0.4 + 0.3j])
def test_pbem_halfspace_matvec_equals_dense_oracle(case, beta):
    counts, L, plane, h = CASES[case]
    v, t = icosphere(1, 0.2)
    k = 3.5
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_PBEM, beta=beta, plane=plane)
    assert op.info["halfspace"] == 1 and op.info["hankel_axis"] == h
    assert op.info["image_separate"] == (1 if h >= 0 else 0)
    x = random_complex_vectors(31, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    A = hs.dense_matrix_halfspace(v, t, L, counts, k, hs.Plane(*plane), beta)
    assert _rel(y, x @ A.T) < 1e-12


@pytest.mark.parametrize("case", ["parallel", "perpendicular"])
def test_pbem_halfspace_fp32_matvec(case):
    counts, L, plane, h = CASES[case]
    v, t = icosphere(1, 0.2)
    op = gb.Operator(v, t, counts, L, 3.5, form=gb.FORM_PBEM, precision=gb.FP32, plane=plane)
    x = random_complex_vectors(32, 3, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    A = hs.dense_matrix_halfspace(v, t, L, counts, 3.5, hs.Plane(*plane))
    assert _rel(y, x @ A.T) < 1e-5


FMM_CASE = ((3, 1, 4), np.diag([0.7, 1.0, 0.7]), (2, -0.45, 0.9 + 0.2j))


@pytest.mark.parametrize("precision,tol", [("FP64", 1e-12), ("FP32", 1e-5)])
def test_fmm_halfspace_matvec_equals_explicit_oracle(precision, tol):
    counts, L, plane = FMM_CASE
    v, t = icosphere(1, 0.2)
    k, nt = 2.0, 6
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_FMM, n_t=nt, precision=getattr(gb, precision), plane=plane)
    pl = hs.Plane(*plane)
    assert op.info["form_name"] == "fmm" and op.info["n_near_image"] == len(hs.image_near_offsets(L, counts, pl))
    x = random_complex_vectors(33, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    cell = bem.CellMesh(v, t)
    ref = fmm.fmm_matvec_explicit(cell, L, counts, k, nt, x) + hs.fmm_image_matvec_explicit(cell, L, counts, k, nt,
                                                                                            pl, x)
    assert _rel(y, ref) < tol


def test_fmm_halfspace_parallel_lattice_and_admittance():
    # lattice parallel to the plane: the image part still has its own tables
    v, t = icosphere(1, 0.2)
    counts, L, plane, k, nt, beta = (4, 3, 1), np.diag([0.7, 0.7, 1.0]), (2, -0.5, -1.0), 2.5, 6, 0.3 + 0.2j
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_FMM, n_t=nt, beta=beta, plane=plane)
    assert op.info["hankel_axis"] == -1 and op.info["image_separate"] == 1
    x = random_complex_vectors(34, 1, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    cell = bem.CellMesh(v, t)
    pl = hs.Plane(*plane)
    ref = (fmm.fmm_matvec_explicit(cell, L, counts, k, nt, x, beta=beta)
           + hs.fmm_image_matvec_explicit(cell, L, counts, k, nt, pl, x, beta=beta))
    assert _rel(y, ref) < 1e-12


@pytest.mark.parametrize("kind,vec", [("plane", [0.48, 0.6, -0.64]), ("monopole", [1.3, -0.4, 0.9])])
def test_incident_rhs_and_field_points_match_oracle(kind, vec):
    counts, L, plane, h = CASES["perpendicular"]
    v, t = icosphere(1, 0.2)
    k = 2.0
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_PBEM, plane=plane, beta=0.2 + 0.1j)
    pl = hs.Plane(*plane)
    cell = bem.CellMesh(v, t)
    inc = [(kind, vec, 1.0), (kind, vec, 0.5 - 0.25j)]
    b = op.rhs_incident(inc).cpu().numpy()
    for r in range(2):
        assert _rel(b[r], hs.rhs(cell, L, counts, k, kind, vec, inc[r][2], pl)) < 1e-13
    p = random_complex_vectors(35, 2, op.N)
    # far, near and very-near points, all above the plane z = -0.26
    pts = np.array([[0.35, 0.1, 0.05], [-0.3, 0.2, 0.1], [0.25, 0.0, 0.62], [1.5, -0.5, 0.3], [0.22, 0.0, 0.0],
                    [0.1, 0.1, -0.2]])
    out = op.field_incident(_dev(p), inc, pts).cpu().numpy()
    for r in range(2):
        ref = hs.field_points(v, t, L, counts, k, p[r], pts, kind, vec, inc[r][2], pl, beta=0.2 + 0.1j)
        assert _rel(out[r], ref) < 1e-12


def test_plane_wave_rhs_of_a_halfspace_operator_includes_the_reflected_wave():
    counts, L, plane, h = CASES["parallel"]
    v, t = icosphere(0, 0.2)
    op = gb.Operator(v, t, counts, L, 2.0, form=gb.FORM_PBEM, plane=plane)
    d = [0.6, 0.0, -0.8]
    b = op.rhs_plane_wave([d]).cpu().numpy()[0]
    ref = hs.rhs(bem.CellMesh(v, t), L, counts, 2.0, "plane", d, 1.0, hs.Plane(*plane))
    assert _rel(b, ref) < 1e-13


def test_pbem_halfspace_solve_matches_dense_oracle():
    counts, L, plane, h = CASES["perpendicular"]
    v, t = icosphere(1, 0.2)
    k = 3.0
    A = hs.dense_matrix_halfspace(v, t, L, counts, k, hs.Plane(*plane))
    for precision, tol, err in (("FP64", 1e-12, 1e-9), ("MIXED", 1e-11, 1e-8)):
        op = gb.Operator(v, t, counts, L, k, form=gb.FORM_PBEM, plane=plane, precision=getattr(gb, precision))
        b = op.rhs_incident([("monopole", [1.0, 0.3, 0.4], 2.0)])
        p, info = op.solve(b, tol=tol, restart=60)
        pref = np.linalg.solve(A, b.cpu().numpy()[0])
        assert info[0]["converged"]
        assert _rel(p.cpu().numpy()[0], pref) < err, precision


def test_fmm_halfspace_solve_matches_dense_oracle():
    counts, L, plane = FMM_CASE
    v, t = icosphere(1, 0.2)
    k = 2.0
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_FMM, n_t=10, plane=plane)
    b = op.rhs_incident([("plane", [0.6, 0.0, -0.8], 1.0)])
    p, info = op.solve(b, tol=1e-10)
    A = hs.dense_matrix_halfspace(v, t, L, counts, k, hs.Plane(*plane))
    pref = np.linalg.solve(A, b.cpu().numpy()[0])
    assert info[0]["converged"]
    assert _rel(p.cpu().numpy()[0], pref) < 1e-3


def test_halfspace_argument_errors():
    v, t = icosphere(0, 0.2)
    # oblique lattice vector
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, (2, 2, 1), np.array([[0.5, 0, 0.1], [0, 0.5, 0], [0, 0, 1.0]]), 2.0, plane=(2, -0.3, 1.0))
    # cells crossing the plane
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, (2, 1, 1), np.diag([0.5, 1.0, 1.0]), 2.0, plane=(2, 0.1, 1.0))
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, (1, 1, 3), np.diag([1.0, 1.0, -0.5]), 2.0, plane=(2, -0.3, 1.0))
    # BF16 is not offered for half-space operators
    with pytest.raises(gb.FmpbError):
        gb.Operator(v, t, (4, 1, 1), np.diag([0.7, 1.0, 1.0]), 2.0, form=gb.FORM_FMM, precision=gb.BF16,
                    plane=(2, -0.3, 1.0))


class _Rows:
    def __init__(self, cell, rows):
        self.centroid = cell.centroid[rows]
        self.normal = cell.normal[rows]
        self.n = len(rows)


def test_barrier_full_size_sampled_rows():
    """The 3x25x5 cylinder barrier on a rigid ground, N = 126,000, FMM form
    with the block Hankel image part along z: sampled rows against the
    oracle's explicit near + U K V sums of both parts (n_t = 6 instead of the
    workload's 10 keeps the oracle's M2L blocks affordable; sizes, launch
    shapes and the near/far split are the workload's)."""
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    v, t = w.mesh()
    k, nt = w.wavenumbers[1], 6
    op = gb.Operator(v, t, w.counts, w.lattice, k, n_t=nt, plane=w.plane)
    assert op.info["form_name"] == "fmm" and op.info["hankel_axis"] == 2 and op.N == 126000
    x = random_complex_vectors(w.rhs_seed, 1, op.N)[0]
    y = op.matvec(_dev(x[None])).cpu().numpy()[0]
    cell = bem.CellMesh(v, t)
    n, L, counts = cell.n, np.asarray(w.lattice, float), w.counts
    pl = hs.Plane(*w.plane)
    cells = bem.lattice_cells(counts)
    V0 = fmm.p2m_table(cell, k, nt)
    U0 = fmm.l2p_table(cell, k, nt)
    V0h = pl.Rp * fmm.p2m_table(hs.reflected_cell(cell, pl), k, nt)
    q = hs.reverse_cells(x[None], counts, 2)[0]
    Mom = x.reshape(len(cells), n) @ V0.T
    Momh = q.reshape(len(cells), n) @ V0h.T
    near_img = set(hs.image_near_offsets(L, counts, pl))
    rc = hs.reflected_cell(cell, pl)
    m2l = {}

    def K(key, d):
        if key not in m2l:
            m2l[key] = fmm.m2l_block(d, k, nt)
        return m2l[key]

    for c, i in [(0, 5), (3 * 12 + 1 + 75 * 2, 200), (3 * 12 + 1 + 75 * 2, 335)]:
        acc = 0.0 + 0.0j
        loc = np.zeros(V0.shape[0], dtype=complex)
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(cells[c], cp))
            if max(abs(d) for d in delta) <= 1:
                selfp = np.zeros((1, n), dtype=bool)
                if not any(delta):
                    selfp[0, i] = True
                D, H = bem.dh_block(_Rows(cell, [i]), cell.v - np.asarray(delta, float) @ L, k, self_pairs=selfp)
                row = -(D + bem.coupling(k) * H)[0]
                if not any(delta):
                    row[i] += 0.5
                acc += row @ x[cj * n:(cj + 1) * n]
            else:
                loc += K(("d", delta), np.asarray(delta, float) @ L) @ Mom[cj]
            if delta in near_img:
                sh = hs.image_shift(L, counts, pl, delta)
                D, H = bem.dh_block(_Rows(cell, [i]), rc.v + sh, k)
                acc += pl.Rp * (-(D + bem.coupling(k) * H)[0]) @ q[cj * n:(cj + 1) * n]
            else:
                loc += K(("i", delta), -hs.image_shift(L, counts, pl, delta)) @ Momh[cj]
        ref = acc + U0[i] @ loc
        assert abs(y[c * n + i] - ref) <= 1e-11 * abs(ref), (c, i)


def test_insertion_loss_matches_oracle():
    counts, L, plane, h = CASES["perpendicular"]
    v, t = icosphere(1, 0.2)
    k = 2.5
    op = gb.Operator(v, t, counts, L, k, form=gb.FORM_PBEM, plane=plane)
    inc = [("monopole", [-2.0, 0.4, 0.5], 2.0), ("monopole", [-2.0, -0.6, 0.5], 1.0)]
    b = op.rhs_incident(inc)
    p, info = op.solve(b, tol=1e-10, restart=80)
    rng = np.random.default_rng(8)
    pts = np.column_stack([rng.uniform(1.0, 2.0, 40), rng.uniform(-0.5, 0.5, 40), rng.uniform(0.0, 1.0, 40)])
    il = op.insertion_loss(p, inc, pts)
    ref = hs.insertion_loss(v, t, L, counts, k, p.cpu().numpy(), pts, inc, hs.Plane(*plane))
    assert abs(il - ref) < 1e-9
    # no surface response: the total field is the incident field
    assert abs(op.insertion_loss(torch.zeros_like(p), inc, pts)) < 1e-12

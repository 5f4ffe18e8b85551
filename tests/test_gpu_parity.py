"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on seeded inputs that span several tiles and ragged tails.

Tolerances: FP64 path, so 1e-12 relative (L2 or max norm) for products and
tables; solved pressure 1e-3 against the dense exact oracle (the FMM
truncation error), 1e-7 against the same operator's residual.
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm
from workloads import WORKLOADS, icosphere, cube, capped_cylinder, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


# ----------------------------------------------------------- quadrature ---

@pytest.mark.parametrize("mesh,counts,lattice,k", [
    ("ico1", (2, 2, 1), np.diag([0.5, 0.45, 1.0]), 3.0),
    ("cube", (2, 1, 1), np.diag([0.5, 0.5, 0.5]), 6.0),
])
def test_collocation_blocks_match_oracle(mesh, counts, lattice, k):
    v, t = {"ico1": lambda: icosphere(1, 0.2), "cube": lambda: cube(0.3, 4)}[mesh]()
    offs = bem.all_offsets(counts)
    T = gb.build_blocks(v, t, counts, lattice, k, offs).cpu().numpy()
    cell = bem.CellMesh(v, t)
    for o, d in enumerate(offs):
        ref = bem.toeplitz_block(cell, lattice, d, k)
        assert np.abs(T[o] - ref).max() <= 1e-12 * np.abs(ref).max(), d


class _Rows:
    """Target subset of a CellMesh (rows of a block)."""

    def __init__(self, cell, rows):
        self.centroid = cell.centroid[rows]
        self.normal = cell.normal[rows]
        self.n = len(rows)


def _oracle_rows(cell, lattice, counts, k, rows_global, x):
    """y_i = sum_j A_ij x_j for a few global rows, by quadrature row by row."""
    n = cell.n
    cells = bem.lattice_cells(counts)
    L = np.asarray(lattice, dtype=float)
    out = []
    for gi in rows_global:
        c, i = divmod(gi, n)
        tgt = _Rows(cell, [i])
        acc = 0.0 + 0.0j
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(cells[c], cp))
            shift = -np.asarray(delta, dtype=float) @ L
            selfp = np.zeros((1, n), dtype=bool)
            if not any(delta):
                selfp[0, i] = True
            D, H = bem.dh_block(tgt, cell.v + shift, k, self_pairs=selfp)
            row = -(D + bem.coupling(k) * H)[0]
            if not any(delta):
                row[i] += 0.5
            acc += row @ x[cj * n:(cj + 1) * n]
        out.append(acc)
    return np.array(out)


# ------------------------------------------------------------ multipole ---

def test_p2m_l2p_tables_match_oracle():
    v, t = icosphere(1, 0.2)
    k, nt = 2.5, 6
    V0, U0 = gb.multipole_tables(v, t, k, nt)
    cell = bem.CellMesh(v, t)
    assert _rel(V0.cpu().numpy(), fmm.p2m_table(cell, k, nt)) < 1e-12
    assert _rel(U0.cpu().numpy(), fmm.l2p_table(cell, k, nt)) < 1e-12


@pytest.mark.parametrize("nt", [1, 4, 8, 12])
def test_m2l_blocks_match_oracle(nt):
    rng = np.random.default_rng(nt)
    d = rng.normal(size=(5, 3)) * 2.0
    d = np.vstack([d, [[0, 0, 1.7], [0, 0, -2.2], [3.0, 0, 0]]])
    for k in (0.7, 4.0):
        K = gb.m2l_blocks(k, nt, d).cpu().numpy()
        for i in range(len(d)):
            ref = fmm.m2l_block(d[i], k, nt)
            assert _rel(K[i], ref) < 1e-12, (nt, k, i)


# ------------------------------------------------------------ circulant ---

@pytest.mark.parametrize("counts,B,R", [((4, 1, 1), 5, 1), ((3, 2, 1), 7, 3), ((2, 3, 2), 4, 6),
                                        ((5, 4, 1), 33, 2), ((1, 1, 1), 3, 1), ((6, 1, 1), 1, 5)])
def test_circulant_product_equals_explicit_block_toeplitz(counts, B, R):
    offs = bem.all_offsets(counts)
    blocks = random_complex_vectors(1000 + B, len(offs), B * B).reshape(len(offs), B, B)
    ncell = int(np.prod(counts))
    x = random_complex_vectors(2000 + R, R, ncell * B)
    spec = gb.circulant_spectrum(counts, _dev(blocks))
    y = gb.circulant_apply(counts, spec, _dev(x)).cpu().numpy()
    ref = bem.toeplitz_matvec(dict(zip(offs, blocks)), counts, x)
    assert _rel(y, ref) < 1e-12
    y0 = _dev(x)
    gb.circulant_apply(counts, spec, _dev(x), out=y0, accumulate=True)
    assert _rel(y0.cpu().numpy(), ref + x) < 1e-12


@pytest.mark.parametrize("counts,B,R", [((4, 1, 1), 5, 1), ((3, 2, 1), 7, 3), ((2, 3, 2), 4, 6),
                                        ((5, 4, 1), 33, 2), ((1, 1, 1), 3, 1), ((6, 1, 1), 1, 5),
                                        ((16, 1, 3), 9, 9), ((32, 2, 1), 3, 2)])
def test_circulant_f32_product_equals_explicit_block_toeplitz(counts, B, R):
    # FP32 spectrum, FP32 DFT passes and products: within 1e-5 of the exact
    # block Toeplitz product (ragged inner tiles, direct and two-factor
    # passes, R >= 8 through the tiled product)
    offs = bem.all_offsets(counts)
    blocks = random_complex_vectors(1100 + B, len(offs), B * B).reshape(len(offs), B, B)
    ncell = int(np.prod(counts))
    x = random_complex_vectors(2100 + R, R, ncell * B)
    spec = gb.circulant_spectrum(counts, _dev(blocks))
    y = gb.circulant_apply_f32(counts, spec, _dev(x)).cpu().numpy()
    ref = bem.toeplitz_matvec(dict(zip(offs, blocks)), counts, x)
    assert _rel(y, ref) < 1e-5
    y0 = _dev(x)
    gb.circulant_apply_f32(counts, spec, _dev(x), out=y0, accumulate=True)
    assert _rel(y0.cpu().numpy(), ref + x) < 1e-5


@pytest.fixture
def dft_plan(request):
    gb.set_dft_plan(request.param)
    yield request.param
    gb.set_dft_plan(-1)


@pytest.mark.parametrize("dft_plan", [0, 1, 2], indirect=True)
@pytest.mark.parametrize("counts,B,R", [((16, 1, 3), 9, 9), ((16, 2, 1), 5, 3), ((3, 16, 1), 7, 2)])
def test_circulant_f32_every_plan_kind(counts, B, R, dft_plan):
    # every plan kind of the FP32 passes forced in turn, on grids whose 16-cell
    # axes pad to P = 32 (the radix-2 form's length), against the exact product
    offs = bem.all_offsets(counts)
    blocks = random_complex_vectors(1200 + B, len(offs), B * B).reshape(len(offs), B, B)
    ncell = int(np.prod(counts))
    x = random_complex_vectors(2200 + R, R, ncell * B)
    spec = gb.circulant_spectrum(counts, _dev(blocks))
    y = gb.circulant_apply_f32(counts, spec, _dev(x)).cpu().numpy()
    ref = bem.toeplitz_matvec(dict(zip(offs, blocks)), counts, x)
    assert _rel(y, ref) < 1e-5


def test_circulant_long_axis_without_a_short_split():
    # P = 245 = 5 * 7 * 7 has no split into two factors of at most 16: the
    # float-float product takes the direct pass, the FP32 one is refused
    counts, B, R = (123, 1, 1), 2, 1
    offs = bem.all_offsets(counts)
    assert gb.circulant_shape(counts)[0][0] == 245
    blocks = random_complex_vectors(1200, len(offs), B * B).reshape(len(offs), B, B)
    x = random_complex_vectors(2200, R, 123 * B)
    spec = gb.circulant_spectrum(counts, _dev(blocks))
    y = gb.circulant_apply(counts, spec, _dev(x)).cpu().numpy()
    assert _rel(y, bem.toeplitz_matvec(dict(zip(offs, blocks)), counts, x)) < 1e-12
    with pytest.raises(gb.FmpbError):
        gb.circulant_apply_f32(counts, spec, _dev(x))


def test_circulant_spectrum_is_the_dft_of_the_first_block_column():
    counts = (3, 2, 1)
    offs = bem.all_offsets(counts)
    B = 2
    blocks = random_complex_vectors(77, len(offs), B * B).reshape(len(offs), B, B)
    spec = gb.circulant_spectrum(counts, _dev(blocks)).cpu().numpy()
    (Px, Py, Pz), F = gb.circulant_shape(counts)
    # brute-force O(F^2) DFT of c[delta mod P] (Eq. (blockDiagonal))
    ref = np.zeros((F, B, B), dtype=complex)
    for o, (dx, dy, dz) in enumerate(offs):
        for fz in range(Pz):
            for fy in range(Py):
                for fx in range(Px):
                    ph = (fx * (dx % Px) / Px + fy * (dy % Py) / Py + fz * (dz % Pz) / Pz)
                    ref[(fz * Py + fy) * Px + fx] += blocks[o] * np.exp(-2j * np.pi * ph)
    assert _rel(spec, ref) < 1e-13


# ------------------------------------------------------------- operator ---

def test_pbem_operator_matvec_equals_dense_oracle():
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (3, 2, 1), np.diag([0.5, 0.6, 1.0]), 3.0
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM)
    assert op.info["form_name"] == "pbem" and op.info["B"] == 80
    x = random_complex_vectors(11, 3, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    A = bem.dense_matrix(v, t, lattice, counts, k)
    assert _rel(y, x @ A.T) < 1e-12


@pytest.mark.parametrize("name,level,nt", [("sphere_row_4", 2, 6), ("grid2d", 1, 5)])
def test_fmm_operator_matvec_equals_explicit_oracle(name, level, nt):
    if name == "sphere_row_4":
        w = WORKLOADS[name]
        counts, lattice, k = w.counts, w.lattice, w.wavenumbers[0]
    else:
        counts, lattice, k = (5, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0
    v, t = icosphere(level, 0.2)
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt)
    assert op.info["form_name"] == "fmm" and op.info["n_near"] == 3 ** (1 if counts[1] == 1 else 2)
    x = random_complex_vectors(12, 2, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = fmm.fmm_matvec_explicit(bem.CellMesh(v, t), lattice, counts, k, nt, x)
    assert _rel(y, ref) < 1e-12


def test_rhs_and_field_points_match_oracle():
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (2, 1, 1), np.diag([0.7, 1.0, 1.0]), 2.0
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM)
    dirs = np.array([[1.0, 0, 0], [0, 0.6, 0.8]])
    amps = np.array([1.0, 0.5 - 0.25j])
    b = op.rhs_plane_wave(dirs, amps).cpu().numpy()
    cell = bem.CellMesh(v, t)
    for r in range(2):
        ref = bem.plane_wave_rhs(cell, lattice, counts, k, dirs[r], amps[r])
        assert _rel(b[r], ref) < 1e-13
    p = random_complex_vectors(13, 2, op.N)
    pts = np.array([[0.35, 0.1, 0.05], [-0.3, 0.2, 0.1], [0.35, 0.0, 0.45], [1.5, -0.5, 0.3], [0.22, 0.0, 0.0]])
    out = op.field(_dev(p), dirs, pts, amps).cpu().numpy()
    for r in range(2):
        ref = bem.field_points(v, t, lattice, counts, k, p[r], pts, dirs[r], amps[r])
        assert _rel(out[r], ref) < 1e-12


def test_solve_matches_dense_oracle_and_reports_residual():
    w = WORKLOADS["sphere_row_4"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t)
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0.6, 0, -0.8]])
    b = op.rhs_plane_wave(dirs)
    p, info = op.solve(b, tol=1e-10)
    p = p.cpu().numpy()
    A = bem.dense_matrix(v, t, w.lattice, w.counts, k)
    cell = bem.CellMesh(v, t)
    for r in range(3):
        bref = bem.plane_wave_rhs(cell, w.lattice, w.counts, k, dirs[r])
        pref = np.linalg.solve(A, bref)
        assert _rel(p[r], pref) < 1e-3
        assert info[r]["converged"] and info[r]["relres_true"] < 1e-9
    # the same operator's residual, computed by the oracle's explicit FMM product
    Ap = fmm.fmm_matvec_explicit(cell, w.lattice, w.counts, k, w.n_t, p)
    bh = b.cpu().numpy()
    assert _rel(Ap, bh) < 1e-9


def test_pbem_solve_matches_dense_oracle():
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (3, 3, 1), np.diag([0.45, 0.45, 1.0]), 5.0
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM)
    b = op.rhs_plane_wave([[0.8, 0.6, 0.0]])
    p, info = op.solve(b, tol=1e-12, restart=20)
    A = bem.dense_matrix(v, t, lattice, counts, k)
    pref = np.linalg.solve(A, b.cpu().numpy()[0])
    assert _rel(p.cpu().numpy()[0], pref) < 1e-9


def test_solver_failure_statuses_are_reported_without_faults():
    v, t = icosphere(1, 0.2)
    op = gb.Operator(v, t, (3, 1, 1), np.eye(3), 2.0, form=gb.FORM_PBEM)
    b = op.rhs_plane_wave([[1.0, 0, 0]])
    p, info = op.solve(b, tol=1e-14, restart=2, maxit=2, raise_on_noconv=False)
    assert info[0]["iters"] == 2 and not info[0]["converged"]
    with pytest.raises(gb.FmpbError) as e:
        op.solve(b, tol=1e-14, restart=2, maxit=2)
    assert e.value.name == "FMPB_ENOCONV"
    with pytest.raises(gb.FmpbError) as e:
        op.solve(b, tol=1e-300, restart=5, maxit=100000, timeout_ms=30)
    assert e.value.name == "FMPB_ETIMEOUT"
    bad = b.clone()
    bad[0, 7] = float("nan")
    with pytest.raises(gb.FmpbError) as e:
        op.solve(bad)
    assert e.value.name == "FMPB_ENAN"
    with pytest.raises(gb.FmpbError) as e:
        gb.Operator(v, t, (6, 1, 1), np.eye(3) * 0.19, 2.0, form=gb.FORM_FMM)
    assert e.value.name == "FMPB_EADMISS"
    bad_t = t.copy()
    bad_t[3, 1] = 10_000
    with pytest.raises(gb.FmpbError) as e:
        gb.Operator(v, bad_t, (2, 1, 1), np.eye(3), 2.0)
    assert e.value.name == "FMPB_EMESH"


# ------------------------------------------------- full-size sampled rows ---

def test_sonic_crystal_full_size_sampled_rows():
    """3x20 capped cylinders, N = 72,000, PBEM form: sampled rows of A x."""
    w = WORKLOADS["sonic_crystal_3x20"]
    v, t = w.mesh()
    k = w.wavenumbers[2]
    op = gb.Operator(v, t, w.counts, w.lattice, k)
    assert op.info["form_name"] == "pbem" and op.info["P"] == [5, 40, 1]
    x = random_complex_vectors(w.rhs_seed, 1, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()[0]
    rows = [0, 1199, 35 * 1200 + 611, 59 * 1200 + 17, 31 * 1200 + 1187]
    ref = _oracle_rows(bem.CellMesh(v, t), w.lattice, w.counts, k, rows, x[0])
    assert np.abs(y[rows] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_sphere_array_full_size_sampled_rows():
    """32x32 spheres, N = 327,680, FMM form (n_t = 8): sampled rows against the
    oracle's explicit near + U K V sums for those rows."""
    w = WORKLOADS["sphere_array_32x32"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t)
    x = random_complex_vectors(w.rhs_seed, 1, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()[0]
    cell = bem.CellMesh(v, t)
    n, nt = cell.n, w.n_t
    cells = bem.lattice_cells(w.counts)
    V0 = fmm.p2m_table(cell, k, nt)
    U0 = fmm.l2p_table(cell, k, nt)
    Mom = x.reshape(len(cells), n) @ V0.T
    L = np.asarray(w.lattice, dtype=float)
    for c, i in [(0, 5), (33 * 16 + 7, 100), (1023, 319)]:
        acc = 0.0 + 0.0j
        loc = np.zeros(V0.shape[0], dtype=complex)
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(cells[c], cp))
            if max(abs(d) for d in delta) <= 1:
                shift = -np.asarray(delta, dtype=float) @ L
                selfp = np.zeros((1, n), dtype=bool)
                if not any(delta):
                    selfp[0, i] = True
                D, H = bem.dh_block(_Rows(cell, [i]), cell.v + shift, k, self_pairs=selfp)
                row = -(D + bem.coupling(k) * H)[0]
                if not any(delta):
                    row[i] += 0.5
                acc += row @ x[0, cj * n:(cj + 1) * n]
            else:
                loc += fmm.m2l_block(np.asarray(delta, dtype=float) @ L, k, nt) @ Mom[cj]
        ref = acc + U0[i] @ loc
        assert abs(y[c * n + i] - ref) <= 1e-11 * abs(ref), (c, i)


# ---------------------------------------------------------- mixed precision ---

def test_fp32_operator_products_and_mixed_refinement():
    """FP32 spectrum: products within 1e-5 of the FP64 oracle; MIXED operator:
    GMRES-IR (FP32 inner solves, accurate outer residuals) reaches the FP64
    tolerance and the FP64 solution."""
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (4, 3, 1), np.diag([0.5, 0.45, 1.0]), 4.0
    x = random_complex_vectors(31, 2, int(np.prod(counts)) * len(t))
    A = bem.dense_matrix(v, t, lattice, counts, k)
    ref = x @ A.T
    op32 = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, precision=gb.FP32)
    assert op32.info["precision_name"] == "fp32"
    y32 = op32.matvec(_dev(x)).cpu().numpy()
    err32 = _rel(y32, ref)
    assert 1e-9 < err32 < 1e-5
    opm = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, precision=gb.MIXED)
    ym = opm.matvec(_dev(x)).cpu().numpy()
    assert _rel(ym, ref) < 1e-12              # MIXED products use the accurate spectrum
    b = opm.rhs_plane_wave([[0.6, 0.8, 0.0]])
    p, info = opm.solve(b, tol=1e-10, restart=30, inner_tol=1e-4)
    assert info[0]["converged"] and info[0]["refinements"] >= 2 and info[0]["relres_true"] <= 1e-10
    pref = np.linalg.solve(A, b.cpu().numpy()[0])
    assert _rel(p.cpu().numpy()[0], pref) < 1e-8
    p32, info32 = op32.solve(op32.rhs_plane_wave([[0.6, 0.8, 0.0]]), tol=1e-5, restart=30)
    assert _rel(p32.cpu().numpy()[0], pref) < 1e-3


def test_fmm_fp32_operator_products():
    w = WORKLOADS["sphere_row_4"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t, precision=gb.FP32)
    x = random_complex_vectors(32, 1, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    ref = fmm.fmm_matvec_explicit(bem.CellMesh(v, t), w.lattice, w.counts, k, w.n_t, x)
    assert _rel(y, ref) < 1e-5


@pytest.mark.parametrize("R", [9, 35])
def test_many_rhs_products_match_oracle(R):
    """R >= 8 takes the tiled per-frequency GEMM (one pass over the spectrum)."""
    v, t = icosphere(1, 0.2)
    counts, lattice, k = (3, 2, 1), np.diag([0.5, 0.6, 1.0]), 3.0
    A = bem.dense_matrix(v, t, lattice, counts, k)
    x = random_complex_vectors(40 + R, R, A.shape[0])
    ref = x @ A.T
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM)
    assert _rel(op.matvec(_dev(x)).cpu().numpy(), ref) < 1e-12
    op32 = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_PBEM, precision=gb.FP32)
    assert _rel(op32.matvec(_dev(x)).cpu().numpy(), ref) < 1e-5


def test_fmm_fp32_many_rhs_products():
    v, t = icosphere(1, 0.2)
    counts, lattice, k, nt = (5, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0, 5
    x = random_complex_vectors(50, 10, int(np.prod(counts)) * len(t))
    ref = fmm.fmm_matvec_explicit(bem.CellMesh(v, t), lattice, counts, k, nt, x)
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt, precision=gb.FP32)
    assert _rel(op.matvec(_dev(x)).cpu().numpy(), ref) < 1e-5
    op64 = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt)
    assert _rel(op64.matvec(_dev(x)).cpu().numpy(), ref) < 1e-12

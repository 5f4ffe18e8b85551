"""Tensor-core (tcgen05, BF16 inputs, FP32 accumulation) products through the C ABI.

fmpb_offset_gemm_bf16 defines its inputs as FP64 -> FP32 -> BF16 roundings
(nearest even at each step), so its result is pinned against the exact
product of those rounded inputs, computed here in FP64: the only difference
left is FP32 accumulation, bounded by about K x 2^-24 relative for K real
terms (K <= 6,000 below, so 1e-5 in the L2 norm is a safe bound).  The
rounding is emulated bit-exactly on the host (round-to-nearest-even on the
FP32 bit pattern).

fmpb_circulant_apply_bf16 runs the per-frequency products Lambda_f X_f of the
circulant engine on the tensor cores; it is pinned against numpy's FFT of the
zero-padded grid, the same BF16 rounding of Lambda_f and X_f, the FP64
product and the inverse FFT with crop (an arbitrary spectrum defines a valid
circulant product, so random spectra serve).

The BF16 operator is checked against the oracle's explicit FMM operator:
two roundings of relative size <= 2^-8 per product term give a product
error of a few 1e-3, so the bound is 1e-2 (and at least 1e-4, to show the
BF16 path actually ran).  GMRES-IR with BF16 inner products must still
reach the FP64 tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import bem, fmm
from workloads import WORKLOADS, icosphere, random_complex_vectors

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _bf16(a):
    """FP64 -> FP32 (nearest) -> BF16 (nearest even), returned as float64 values."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _cbf16(z):
    return _bf16(z.real) + 1j * _bf16(z.imag)


def _reference(counts, offsets, T, x):
    """y[r, c] = sum_o T[o] x[r, c - delta_o] over cells inside the grid (FP64)."""
    Mx, My, Mz = counts
    Nc = Mx * My * Mz
    R = x.shape[0]
    n_off, m, k = T.shape
    xc = x.reshape(R, Nc, k)
    y = np.zeros((R, Nc, m), dtype=np.complex128)
    c = np.arange(Nc)
    cx, cy, cz = c % Mx, (c // Mx) % My, c // (Mx * My)
    for o, (dx, dy, dz) in enumerate(offsets):
        sx, sy, sz = cx - dx, cy - dy, cz - dz
        ok = (sx >= 0) & (sx < Mx) & (sy >= 0) & (sy < My) & (sz >= 0) & (sz < Mz)
        src = (sz * My + sy) * Mx + sx
        y[:, ok, :] += xc[:, src[ok], :] @ T[o].T
    return y.reshape(R, Nc * m)


def _case(seed, counts, offsets, m, k, R):
    rng = np.random.default_rng(seed)
    n_off = len(offsets)
    T = (rng.standard_normal((n_off, m, k)) + 1j * rng.standard_normal((n_off, m, k))) * \
        np.exp(rng.uniform(-3, 3, (n_off, 1, 1)))
    Nc = int(np.prod(counts))
    x = random_complex_vectors(seed, R, Nc * k)
    return T, x


OFF27 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
OFF9 = [(dx, dy, 0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


@pytest.fixture
def tile_variant(request):
    gb.set_tile_variant(request.param)
    yield request.param
    gb.set_tile_variant(-1)


@pytest.mark.parametrize("tile_variant", [-1, 0, 1, 2, 3], indirect=True)
@pytest.mark.parametrize("counts,offsets,m,k,R", [
    ((5, 4, 3), OFF27, 20, 20, 3),          # one ragged tile in M, N and K
    ((16, 12, 1), OFF9, 300, 150, 2),       # 5 M tiles (odd: a half-empty 256-row tile), 2 N tiles, 45 K steps
    ((7, 1, 1), [(0, 0, 0)], 81, 320, 5),   # P2M shape, one offset
    ((3, 3, 2), [(0, 0, 0)], 100, 49, 40),  # L2P shape, ragged depth
])
def test_offset_gemm_equals_product_of_rounded_inputs(counts, offsets, m, k, R, tile_variant):
    T, x = _case(7 + m + k, counts, offsets, m, k, R)
    y = gb.offset_gemm_bf16(counts, offsets, _dev(T), _dev(x)).cpu().numpy()
    ref = _reference(counts, offsets, _cbf16(T), _cbf16(x))
    err = _rel(y, ref)
    assert err < 1e-5, err
    # and it is the rounded product, not the exact one
    exact = _reference(counts, offsets, T, x)
    assert _rel(y, exact) > 10 * err


def test_autotuner_records_its_choice():
    T, x = _case(5, (6, 5, 1), OFF9, 64, 40, 3)
    gb.offset_gemm_bf16((6, 5, 1), OFF9, _dev(T), _dev(x))
    entries = [e for e in gb.tuning_summary()
               if e.get("kernel") == "tc_gemm" and (e["m"], e["k"], e["columns"], e["offsets"]) == (64, 40, 90, 9)]
    assert len(entries) == 1
    e = entries[0]
    assert e["rows_per_cta"] in (128, 256) and e["columns_per_cta"] in (128, 256) and len(e["ms"]) == 4
    assert all(t > 0 for t in e["ms"])


@pytest.mark.parametrize("tile_variant", [0, 1, 2, 3], indirect=True)
def test_offset_gemm_accumulates_and_skips_cells_outside_the_grid(tile_variant):
    counts, m, k, R = (4, 3, 2), 33, 17, 2
    offsets = [(1, 0, 0), (-1, 1, 1), (0, 0, -1), (2, 0, 0)]   # the last has sources only for c_x >= 2
    T, x = _case(99, counts, offsets, m, k, R)
    y0 = random_complex_vectors(5, R, int(np.prod(counts)) * m)
    y = gb.offset_gemm_bf16(counts, offsets, _dev(T), _dev(x), out=_dev(y0.copy()), accumulate=True).cpu().numpy()
    ref = y0 + _reference(counts, offsets, _cbf16(T), _cbf16(x))
    assert _rel(y, ref) < 1e-5
    only_outside = gb.offset_gemm_bf16(counts, [(4, 0, 0)], _dev(T[:1]), _dev(x)).cpu().numpy()
    assert np.abs(only_outside).max() == 0.0


@pytest.mark.parametrize("tile_variant", [-1, 0, 1, 2, 3], indirect=True)
@pytest.mark.parametrize("counts,offsets,m,k,k2,R,accumulate", [
    ((5, 4, 3), OFF27, 20, 20, 9, 3, False),        # ragged M, N and K; a one-step tail
    ((16, 12, 1), OFF9, 300, 150, 81, 2, True),     # half-empty 256-row tile, a three-step tail
    ((4, 3, 2), [(1, 0, 0), (-1, 1, 1), (2, 0, 0)], 33, 17, 40, 2, False),   # sources outside the grid
])
def test_offset_gemm_with_tail_equals_product_of_rounded_inputs(counts, offsets, m, k, k2, R, accumulate,
                                                                tile_variant):
    # the FMM product's near field plus L2P term in one accumulation:
    # y = sum_o T_o x_{c - delta_o} + T2 x2_c
    T, x = _case(11 + m + k2, counts, offsets, m, k, R)
    T2, x2 = _case(13 + k2, counts, [(0, 0, 0)], m, k2, R)
    Nc = int(np.prod(counts))
    y0 = random_complex_vectors(17, R, Nc * m) if accumulate else np.zeros((R, Nc * m), dtype=np.complex128)
    y = gb.offset_gemm2_bf16(counts, offsets, _dev(T), _dev(x), _dev(T2[0]), _dev(x2), out=_dev(y0.copy()),
                             accumulate=accumulate).cpu().numpy()
    ref = y0 + _reference(counts, offsets, _cbf16(T), _cbf16(x)) + \
        _reference(counts, [(0, 0, 0)], _cbf16(T2), _cbf16(x2))
    err = _rel(y, ref)
    assert err < 1e-5, err
    with pytest.raises(ValueError):
        gb.offset_gemm2_bf16(counts, offsets, _dev(T), _dev(x), _dev(T2[0, :-1]), _dev(x2))


@pytest.mark.parametrize("counts,B,R", [((3, 4, 1), 40, 70), ((2, 3, 2), 81, 5), ((5, 1, 1), 169, 64),
                                          ((2, 2, 1), 30, 300)])
def test_circulant_bf16_equals_rounded_frequency_products(counts, B, R):
    rng = np.random.default_rng(B + R)
    P, F = gb.circulant_shape(counts)
    Mx, My, Mz = counts
    Px, Py, Pz = P
    spec = rng.standard_normal((F, B, B)) + 1j * rng.standard_normal((F, B, B))
    x = random_complex_vectors(B + R, R, Mx * My * Mz * B)
    y = gb.circulant_apply_bf16(counts, _dev(spec), _dev(x)).cpu().numpy()
    xg = np.zeros((R, Pz, Py, Px, B), dtype=np.complex128)
    xg[:, :Mz, :My, :Mx, :] = x.reshape(R, Mz, My, Mx, B)
    X = np.fft.fftn(xg, axes=(1, 2, 3)).reshape(R, F, B)
    Yf = np.einsum("fij,rfj->rfi", _cbf16(spec), _cbf16(X))
    ref = np.fft.ifftn(Yf.reshape(R, Pz, Py, Px, B), axes=(1, 2, 3))[:, :Mz, :My, :Mx, :].reshape(R, -1)
    err = _rel(y, ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("name,level,nt,counts", [
    ("sphere_row_4", 2, 6, None),
    ("grid2d", 1, 5, (5, 4, 1)),
    ("grid3d", 1, 4, (3, 3, 3)),
])
def test_bf16_operator_matvec_against_explicit_oracle(name, level, nt, counts):
    if name == "sphere_row_4":
        w = WORKLOADS[name]
        counts, lattice, k = w.counts, w.lattice, w.wavenumbers[0]
    else:
        lattice, k = np.diag([0.6, 0.6, 0.6]), 4.0
    v, t = icosphere(level, 0.2)
    op = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt, precision=gb.BF16)
    assert op.info["precision_name"] == "bf16"
    x = random_complex_vectors(61, 3, op.N)
    y = op.matvec(_dev(x)).cpu().numpy()
    op.check()
    ref = fmm.fmm_matvec_explicit(bem.CellMesh(v, t), lattice, counts, k, nt, x)
    err = _rel(y, ref)
    assert 1e-4 < err < 1e-2, err


def test_bf16_requires_the_fmm_form():
    w = WORKLOADS["sonic_crystal_3x20"]
    v, t = w.mesh()
    with pytest.raises(gb.FmpbError) as e:
        gb.Operator(v, t, (3, 2, 1), w.lattice, w.wavenumbers[0], precision=gb.BF16)
    assert e.value.name == "FMPB_EINVAL"


def test_mixed_fmm_refines_bf16_inner_solves_to_fp64_tolerance():
    v, t = icosphere(1, 0.2)
    counts, lattice, k, nt = (5, 4, 1), np.diag([0.6, 0.6, 1.0]), 4.0, 5
    op64 = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt)
    opm = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt, precision=gb.MIXED)
    x = random_complex_vectors(62, 2, op64.N)
    assert _rel(opm.matvec(_dev(x)).cpu().numpy(), op64.matvec(_dev(x)).cpu().numpy()) < 1e-12
    b = op64.rhs_plane_wave([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0]])
    p64, i64 = op64.solve(b, tol=1e-10, restart=60)
    pm, im = opm.solve(b, tol=1e-10, restart=60, inner_tol=1e-2)
    for r in range(2):
        assert im[r]["converged"] and im[r]["relres_true"] <= 1e-10 and im[r]["refinements"] >= 2, im[r]
    assert _rel(pm.cpu().numpy(), p64.cpu().numpy()) < 1e-8
    opb = gb.Operator(v, t, counts, lattice, k, form=gb.FORM_FMM, n_t=nt, precision=gb.BF16)
    pb, ib = opb.solve(b, tol=1e-3, restart=60)
    errb = _rel(pb.cpu().numpy(), p64.cpu().numpy())
    assert errb < 2e-2, errb

"""Pins of the oracle's single-level FMM operators (Sec. 3.1-3.2, Appendix A):
the truncated expansion of G (Eq. (greenFMM)) and of its normal derivatives
must reproduce the kernels, the Wigner-3j M2L (Eqs. (m2l), (wigner)) must
equal an independent projection construction and obey reciprocity and the
axial selection rule, and the explicit FMPBEM operator S + U K V must tend to
the exact block Toeplitz operator as the truncation number grows (the
error-versus-truncation trend of the accuracy study in Sec. 4.1)."""
import numpy as np
import pytest

from oracle import bem, fmm
from oracle import special as sp
from workloads import WORKLOADS, icosphere, random_complex_vectors


def _fac(nt):
    return np.array([2 * n + 1 for n, m in sp.coeff_list(nt)], dtype=float)


def test_multipole_expansion_reproduces_G_and_converges():
    rng = np.random.default_rng(7)
    k = 4.0
    y = rng.normal(size=3)
    y *= 0.4 / np.linalg.norm(y)                # |y - y_c| / |x - y_c| ~ 0.3
    x = np.array([1.1, -0.4, 0.7])
    r = np.linalg.norm(x - y)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    errs = []
    for nt in (4, 8, 12, 16, 25):
        s = 1j * k / (4 * np.pi) * np.sum(_fac(nt) * sp.wave_table(nt, x, k, "O")
                                          * np.conj(sp.wave_table(nt, y, k, "I")))
        errs.append(abs(s - G) / abs(G))
    assert all(b < 0.1 * a for a, b in zip(errs[:4], errs[1:4]))
    assert errs[-1] < 1e-12


def test_normal_derivative_expansions_through_m2l_reproduce_kernels():
    """dG/dn_y (P2M derivative) and d2G/dn_x dn_y (P2M + M2L + L2P derivative)."""
    rng = np.random.default_rng(8)
    k, nt = 3.0, 14
    yc, xc = np.zeros(3), np.array([1.5, 0.3, -0.6])
    y = yc + rng.normal(size=3) * 0.1
    x = xc + rng.normal(size=3) * 0.1
    ny, nx = rng.normal(size=3), rng.normal(size=3)
    ny /= np.linalg.norm(ny)
    nx /= np.linalg.norm(nx)
    f = _fac(nt)
    dIy = np.conj(np.einsum("qi,i->q", sp.grad_regular_table(nt, y - yc, k), ny))   # d conj(I)/dn_y
    dlp = bem.kernel_dlp(x, nx, y, ny, k)
    expand = 1j * k / (4 * np.pi) * np.sum(f * sp.wave_table(nt, x - yc, k, "O") * dIy)
    assert abs(expand - dlp) < 1e-10 * abs(dlp)
    L = fmm.m2l_block(xc - yc, k, nt) @ dIy
    dIx = np.conj(np.einsum("qi,i->q", sp.grad_regular_table(nt, x - xc, k), nx))
    hyp = bem.kernel_hyp(x, nx, y, ny, k)
    local = 1j * k / (4 * np.pi) * np.sum(f * dIx * L)
    assert abs(local - hyp) < 1e-8 * abs(hyp)


@pytest.mark.parametrize("d", [(1.3, -0.7, 0.9), (0.0, 0.0, 2.0), (-2.0, 0.3, 0.0), (0.6, 0.6, 0.0)])
def test_wigner_m2l_equals_projection_m2l(d):
    d = np.array(d)
    K = fmm.m2l_block(d, 2.5, 6)
    Kp = fmm.m2l_block_by_projection(d, 2.5, 6, rho0=0.35 * np.linalg.norm(d))
    assert np.abs(K - Kp).max() < 1e-10 * np.abs(K).max()


def test_m2l_reciprocity_parity_and_axial_selection_rule():
    nt, k = 6, 2.0
    f = _fac(nt)
    d = np.array([1.3, -0.7, 0.9])
    A = fmm.m2l_block(d, k, nt) / f[None, :]
    Am = fmm.m2l_block(-d, k, nt) / f[None, :]
    # G(x, y) = G(y, x): translating the other way is the transpose
    assert np.abs(Am - A.T).max() < 1e-13 * np.abs(A).max()
    par = np.array([[(-1) ** (n + n2) for n2, m2 in sp.coeff_list(nt)] for n, m in sp.coeff_list(nt)])
    assert np.abs(Am - par * A).max() < 1e-13 * np.abs(A).max()
    Kz = fmm.m2l_block(np.array([0.0, 0.0, 2.0]), k, nt)
    for i, (n, m) in enumerate(sp.coeff_list(nt)):
        for j, (n2, m2) in enumerate(sp.coeff_list(nt)):
            if m + m2 != 0:
                assert Kz[i, j] == 0.0


def test_explicit_fmm_operator_tends_to_exact_operator():
    w = WORKLOADS["sphere_row_4"]
    v, t = icosphere(1, 0.2)                    # 80 triangles keep the CPU suite short
    cell = bem.CellMesh(v, t)
    k, counts, L = w.wavenumbers[0], w.counts, w.lattice
    p = random_complex_vectors(w.rhs_seed, 1, cell.n * 4)[0]
    blocks = {d: bem.toeplitz_block(cell, L, d, k) for d in bem.all_offsets(counts)}
    y_exact = bem.toeplitz_matvec(blocks, counts, p)[0]
    near = {d: blocks[d] for d in bem.near_offsets(counts)}
    errs = []
    for nt in (2, 4, 6, 8, 10):
        y = fmm.fmm_matvec_explicit(cell, L, counts, k, nt, p, near_blocks=dict(near))[0]
        errs.append(np.linalg.norm(y - y_exact) / np.linalg.norm(y_exact))
    assert all(b < 0.1 * a for a, b in zip(errs, errs[1:]))
    assert errs[2] < 1e-8 and errs[-1] < 1e-12


# ------------------------------------------------------ truncation rule --

def test_nearest_far_offset_by_hand():
    # 4 x 3 cells at 0.6 x 0.5 m: the shortest far translation is two cells
    # along y (1.0 m; two along x is 1.2 m, a knight's move sqrt(0.36 + 1))
    assert fmm.nearest_far_offset(np.diag([0.6, 0.5, 1.0]), (4, 3, 1)) == (0, -2, 0)
    assert fmm.nearest_far_offset(np.diag([0.4, 0.7, 1.0]), (5, 5, 1)) == (-2, 0, 0)
    assert fmm.nearest_far_offset(np.eye(3), (2, 2, 2)) is None          # every pair is near
    d = fmm.nearest_far_offset(np.diag([1.0, 1.0, 0.45]), (3, 3, 4))
    assert d == (0, 0, -2)


def test_probe_vectors_are_unit_and_spread():
    X = fmm.probe_vectors(257)
    assert np.allclose(np.abs(X), 1.0, atol=1e-15) and np.allclose(X[:, 0], 1.0)
    phi = (np.sqrt(5.0) - 1.0) / 2.0
    assert np.isclose(X[2, 5], np.exp(2j * np.pi * ((3 * 5 * phi) % 1.0)), atol=1e-14)
    G = X.conj() @ X.T / 257                  # the four probes are nearly orthogonal
    assert np.abs(G - np.diag(np.diag(G))).max() < 0.05


@pytest.fixture(scope="module")
def sphere_cell():
    v, t = icosphere(1, 0.2)
    return bem.CellMesh(v, t)


def test_truncation_rule_tracks_the_block_error(sphere_cell):
    # the probe error falls geometrically with n_t, and at the n_t the rule
    # picks the whole block's Frobenius error (no probes) is below 1e-5 while
    # two orders less leave it above 1e-6
    L, counts, k = np.diag([0.6, 0.6, 1.0]), (4, 4, 1), 4.0
    d, errs = fmm.truncation_errors(sphere_cell, L, counts, k, nt_max=14)
    assert d == (0, -2, 0)
    e = [errs[n] for n in range(4, 15)]
    assert all(b < 0.7 * a for a, b in zip(e, e[1:])), e
    nt = fmm.auto_truncation(sphere_cell, L, counts, k, nt_max=14)
    assert errs[nt] <= 1e-6 < errs[nt - 1]
    T = bem.toeplitz_block(sphere_cell, L, d, k)
    dv = np.asarray(d, dtype=float) @ L

    def block_err(n):
        UKV = fmm.l2p_table(sphere_cell, k, n) @ fmm.m2l_block(dv, k, n) @ fmm.p2m_table(sphere_cell, k, n)
        return np.linalg.norm(UKV - T) / np.linalg.norm(T)

    assert block_err(nt) < 1e-5 and block_err(nt - 2) > 1e-6


def test_truncation_rule_grows_with_frequency_and_keeps_the_operator_accurate(sphere_cell):
    # the accuracy study's trend (Sec. 4): higher frequency needs more
    # terms; the whole FMPBEM product at the chosen n_t stays within 1e-5 of
    # the exact block Toeplitz product
    L, counts = np.diag([0.6, 0.6, 1.0]), (4, 3, 1)
    nts = [fmm.auto_truncation(sphere_cell, L, counts, k, nt_max=14) for k in (4.0, 12.0, 20.0)]
    assert nts[0] <= nts[1] <= nts[2] and nts[0] < nts[2], nts
    k, nt = 12.0, nts[1]
    blocks = {d: bem.toeplitz_block(sphere_cell, L, d, k) for d in bem.all_offsets(counts)}
    x = random_complex_vectors(71, 1, sphere_cell.n * 12)
    exact = bem.toeplitz_matvec(blocks, counts, x)
    near = {d: b for d, b in blocks.items() if max(abs(c) for c in d) <= 1}
    y = fmm.fmm_matvec_explicit(sphere_cell, L, counts, k, nt, x, near_blocks=near)
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 1e-5

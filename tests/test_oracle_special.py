"""Pins of the oracle's special functions (Sec. 3.1 Eq. (Onm), Appendix A
Eq. (wigner)) against closed forms, identities and an independent library."""
import numpy as np
import pytest
from scipy.special import lpmv, eval_legendre

from oracle import special as sp


def test_spherical_bessel_closed_forms_and_wronskian():
    x = np.array([0.3, 1.0, 2.7, 7.5, 19.0])
    assert np.allclose(sp.sph_jn(0, x), np.sin(x) / x, rtol=1e-14)
    assert np.allclose(sp.sph_jn(1, x), np.sin(x) / x**2 - np.cos(x) / x, rtol=1e-13)
    h0 = sp.sph_hn(0, x)
    assert np.allclose(h0, np.exp(1j * x) / (1j * x), rtol=1e-14)      # h_0 = e^{ix}/(ix)
    h1 = sp.sph_hn(1, x)
    assert np.allclose(h1, -np.exp(1j * x) * (x + 1j) / x**2, rtol=1e-13)
    for n in range(0, 12):
        # j_n h_n' - j_n' h_n = i / x^2
        w = sp.sph_jn(n, x) * sp.sph_hn_deriv(n, x) - sp.sph_jn_deriv(n, x) * sp.sph_hn(n, x)
        assert np.allclose(w, 1j / x**2, rtol=1e-9)


def test_legendre_against_scipy_and_poles():
    x = np.linspace(-1, 1, 41)
    P = sp.assoc_legendre_table(10, x)
    for n in range(11):
        for m in range(n + 1):
            # scipy's lpmv carries the Condon-Shortley phase (-1)^m
            assert np.allclose(P[n][m], (-1) ** m * lpmv(m, n, x), rtol=1e-12, atol=1e-12)
        assert np.allclose(P[n][0], eval_legendre(n, x), atol=1e-13)
    Q = sp.legendre_over_sin_table(10, x)
    s = np.sqrt(1 - x * x)
    inner = s > 1e-3
    for n in range(1, 11):
        for m in range(1, n + 1):
            assert np.allclose(Q[n][m][inner] * s[inner], P[n][m][inner], rtol=1e-12, atol=1e-13)
            # finite at the poles: Q_n^1(+-1) = P_n'(+-1) up to sign
            assert np.all(np.isfinite(Q[n][m]))


def _rand_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_addition_theorem_and_negative_order():
    rng = np.random.default_rng(1)
    a, b = _rand_unit(rng, 7), _rand_unit(rng, 7)
    nmax = 9
    Ya, Yb = sp.sph_harm_table(nmax, a), sp.sph_harm_table(nmax, b)
    cosg = np.einsum("ij,ij->i", a, b)
    for n in range(nmax + 1):
        s = sum(Ya[sp.coeff_index(n, m)] * np.conj(Yb[sp.coeff_index(n, m)]) for m in range(-n, n + 1))
        assert np.allclose(s, eval_legendre(n, cosg), atol=1e-13)
        for m in range(1, n + 1):
            # Rodrigues convention: Y_n^{-m} = (-1)^m conj(Y_n^m)
            assert np.allclose(Ya[sp.coeff_index(n, -m)], (-1) ** m * np.conj(Ya[sp.coeff_index(n, m)]), atol=1e-14)


def test_orthogonality_of_Y():
    nq = 24
    x, wx = np.polynomial.legendre.leggauss(nq)
    phi = 2 * np.pi * np.arange(2 * nq) / (2 * nq)
    st = np.sqrt(1 - x * x)
    U = np.stack([st[:, None] * np.cos(phi), st[:, None] * np.sin(phi), x[:, None] * np.ones_like(phi)], -1).reshape(-1, 3)
    W = (wx[:, None] * np.full(2 * nq, np.pi / nq)).ravel()
    Y = sp.sph_harm_table(6, U)
    G = (Y * W) @ np.conj(Y).T
    expect = np.diag([4 * np.pi / (2 * n + 1) for n, m in sp.coeff_list(6)])
    assert np.allclose(G, expect, atol=1e-12)


def test_regular_wave_gradient_against_finite_differences():
    rng = np.random.default_rng(2)
    k = 3.1
    pts = rng.normal(size=(6, 3)) * 0.4
    pts = np.vstack([pts, [[0, 0, 0.3], [0, 0, -0.2], [1e-9, 0, 0.25]]])   # on and near the polar axis
    g = sp.grad_regular_table(7, pts, k)
    h = 1e-5
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (sp.wave_table(7, pts + e, k, "I") - sp.wave_table(7, pts - e, k, "I")) / (2 * h)
        assert np.allclose(g[..., ax], fd, atol=2e-8)
    g0 = sp.grad_regular_table(3, np.zeros((1, 3)), k)
    fd0 = np.stack([(sp.wave_table(3, np.eye(3)[a][None] * 1e-6, k, "I")
                     - sp.wave_table(3, -np.eye(3)[a][None] * 1e-6, k, "I")) / 2e-6 for a in range(3)], -1)
    assert np.allclose(g0, fd0, atol=1e-9)


def test_wigner3j_against_sympy_exact_and_orthogonality():
    wig = pytest.importorskip("sympy.physics.wigner")
    cases = [(1, 1, 0, 0, 0, 0), (2, 1, 1, 0, 0, 0), (3, 2, 1, 1, -1, 0), (5, 4, 3, -2, 1, 1),
             (6, 6, 8, 3, -4, 1), (7, 5, 4, 0, 0, 0), (10, 8, 12, -5, 2, 3), (12, 12, 20, 7, -7, 0)]
    for c in cases:
        assert sp.wigner3j(*c) == pytest.approx(float(wig.wigner_3j(*c)), rel=1e-13, abs=1e-16)
    # sum over m1, m2 at fixed m3 = -m1-m2: delta_{j3 j3'} / (2 j3 + 1)
    j1, j2, m3 = 4, 3, 1
    for j3 in range(1, 8):
        for j3b in range(1, 8):
            s = 0.0
            for m1 in range(-j1, j1 + 1):
                m2 = -m1 - m3
                if abs(m2) <= j2:
                    s += sp.wigner3j(j1, j2, j3, m1, m2, m3) * sp.wigner3j(j1, j2, j3b, m1, m2, m3)
            ok = abs(j1 - j2) <= j3 <= j1 + j2 and abs(m3) <= j3
            expect = (1.0 / (2 * j3 + 1)) if (j3 == j3b and ok) else 0.0
            assert s == pytest.approx(expect, abs=1e-14)

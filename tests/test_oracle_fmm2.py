"""Pins of the oracle's FMPBEM2 near-field operator (Sec. 3.3, Eqs. (m2m),
(l2l)):

* the regular translation R by projection satisfies the addition theorem
  I_q(a + b) = sum_q' R_qq'(b) I_q'(a) at points (up to the truncation);
* R equals the 3j form: the coefficient table of Eq. (m2l) evaluated with
  I_l instead of O_l, R[q', (n, -m)] = (-1)^m (2n+1)/(2n'+1) K_reg[(n, m), q']
  (the form the GPU library evaluates);
* M2M of a child's P2M moments converges to the P2M moments about the parent
  centre, and L2P of the child after L2L to the parent's L2P, as n_t grows;
* with no subdivision the near block is the exact one, and every multilevel
  near block converges to the exact S_delta as n_t,near grows.
"""
import numpy as np
import pytest

from oracle import bem, fmm, fmm2, special as sp
from workloads import icosphere


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_regular_translation_is_the_addition_theorem():
    k, nt = 3.0, 12
    rng = np.random.default_rng(7)
    for _ in range(3):
        b = rng.normal(size=3) * 0.1
        a = rng.normal(size=3) * 0.03
        R = fmm2.regular_translation(b, k, nt)
        lhs = sp.wave_table(nt, a + b, k, "I")[:16]
        rhs = (R @ sp.wave_table(nt, a, k, "I"))[:16]
        assert np.abs(lhs - rhs).max() < 1e-10


def test_regular_translation_equals_the_3j_form():
    k, nt = 2.3, 5
    B = (nt + 1) ** 2
    coeffs = sp.coeff_list(nt)
    ent, oidx, coef = fmm._m2l_terms(nt)
    for b in ([0.21, -0.13, 0.17], [0.0, 0.0, 0.3], [-0.1, 0.05, 0.0]):
        Ireg = sp.wave_table(2 * nt, np.asarray(b), k, "I")
        K = np.zeros(B * B, dtype=complex)
        np.add.at(K, ent, coef * Ireg[oidx])
        K = K.reshape(B, B)
        C = np.zeros((B, B), dtype=complex)
        for qi, (n, m) in enumerate(coeffs):
            for qj, (n2, m2) in enumerate(coeffs):
                C[qj, sp.coeff_index(n, -m)] = (-1) ** (m % 2) * (2 * n + 1) / (2 * n2 + 1) * K[qi, qj]
        R = fmm2.regular_translation(np.asarray(b), k, nt)
        assert np.abs(C - R).max() < 1e-12 * np.abs(R).max()


def test_m2m_and_l2l_converge_to_direct_expansions():
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    tree = fmm2.Octree(cell, 1)
    k = 3.0
    child = tree.boxes[1][0]
    el = [j for j, key in enumerate(tree.elem_box[1]) if key == child]
    cc, cp = tree.centre(1, child), tree.centre(0, (0, 0, 0))
    e_m, e_l = [], []
    for nt in (4, 8, 12):
        direct = fmm2.p2m_leaf(cell, el, cp, k, nt)
        shifted = fmm2.m2m_matrix(cc, cp, k, nt) @ fmm2.p2m_leaf(cell, el, cc, k, nt)
        e_m.append(_rel(shifted[:9], direct[:9]))
        Lp = np.random.default_rng(3).normal(size=(nt + 1) ** 2) + 0j
        Lp[9:] = 0.0   # a local expansion of low degree, exactly representable about the child
        up = fmm2.l2p_leaf(cell, el, cp, k, nt) @ Lp
        down = fmm2.l2p_leaf(cell, el, cc, k, nt) @ (fmm2.l2l_matrix(cp, cc, k, nt) @ Lp)
        e_l.append(_rel(down, up))
    # geometric convergence down to rounding
    assert e_m[0] > 100 * e_m[1] and max(e_m[1:]) < 1e-10, e_m
    assert e_l[0] > 100 * e_l[1] and max(e_l[1:]) < 1e-10, e_l


def test_near_blocks_converge_to_the_exact_blocks():
    v, t = icosphere(1, 0.2)
    cell = bem.CellMesh(v, t)
    L, k = np.diag([0.5, 0.55, 1.0]), 3.0
    S0 = bem.toeplitz_block(cell, L, (0, 0, 0), k)
    assert np.array_equal(fmm2.near_block_matrix(cell, fmm2.Octree(cell, 0), L, (0, 0, 0), k, 4, S_exact=S0), S0)
    tree = fmm2.Octree(cell, 2)
    for d in [(0, 0, 0), (1, 0, 0), (-1, 1, 0)]:
        S = bem.toeplitz_block(cell, L, d, k)
        m2l, p2p = fmm2.interaction_lists(tree, -np.asarray(d, float) @ L)
        assert len(m2l) > 0
        errs = [_rel(fmm2.near_block_matrix(cell, tree, L, d, k, nt, S_exact=S), S) for nt in (2, 5, 8)]
        assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-3, (d, errs)

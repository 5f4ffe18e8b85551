"""FMPBEM2 (Sec. 3.3): the unique near blocks S_delta of the FMPBEM are
approximated by a multilevel FMM over an octree of the unit cell, with its
own truncation number n_tn (n_t,near); the interactions between unit cells
stay those of the single-level FMPBEM (fmm.py).  Oracle code: test
infrastructure only.

Octree (the paper: boxes subdivided hierarchically up to a level).  The root
is the cube centred on the midpoint of the bounding box of the element
centroids, with edge e_0 = the longest side of that box times (1 + 1e-9);
level l has boxes of edge e_l = e_0 / 2^l indexed (ix, iy, iz) in
[0, 2^l)^3 (x fastest), and element j belongs to the box containing its
centroid (indices clamped to the last box).  Only occupied boxes exist; the
leaves are the boxes of level L.

Interaction lists per near offset delta (source cell shifted by
s = -delta . L).  Boxes b (target cell) and b' (source cell) of level l are
well separated iff |c_b - (c_b' + s)| >= 3 rho_l (1 - 1e-9), rho_l the
largest distance from a level-l box centre to a vertex of its elements:
Eq. (admissibility), |x_c - y_c| >= 2 r, with r read as 1.5 rho_l, which
keeps the two-centre expansion ratio at 2/3 or less as the cell-level rule
of the FMPBEM does (with r the box edge the ratio reaches 0.87 and a
neighbour cell's whole block becomes one M2L that converges slowly).
Starting from the pair of roots, a well-separated pair is an M2L pair; a
pair that is not is replaced by all pairs of occupied children, or, at level
L, is a P2P pair (the exact entries of S_delta, bem.py).

Expansions of box centres (truncation n_tn, coefficient q = n(n+1) + m):
  P2M of a leaf:  V[q, j] = int_{E_j} conj(dI_q(y - c)/dn_y) dA   (far rule)
  M2M child c_c -> parent c_p (Eq. (m2m)):
       M_q(c_p) = sum_q' conj(R_qq'(c_c - c_p)) M_q'(c_c)
  M2L (Eq. (m2l)): L(c_b) += K(c_b - c_b' - s) M(c_b')            (fmm.m2l_block)
  L2L parent -> child (Eq. (l2l)):
       L_q'(c_c) = sum_q (2n + 1)/(2n' + 1) conj(R_qq'(c_c - c_p)) L_q(c_p)
  L2P of a leaf:  U[i, q] as fmm.l2p_table with the leaf centre
with R the regular translation, I_q(a + b) = sum_q' R_qq'(b) I_q'(a)
(truncated at n_tn).  Eqs. (m2m) and (l2l) are printed with index and sign
patterns that depend on the conjugation convention of the moments; here both
follow from Eq. (greenFMM)'s convention (moments of conj(I), locals against
conj(I)) and the addition theorem, and R is computed by projection on a
sphere, independently of the 3j table.
"""
from functools import lru_cache

import numpy as np

from . import special as sp
from .bem import CellMesh, collapsed_rule, Q_FAR, coupling, toeplitz_block, lattice_cells, near_offsets

TIE = 1e-9


class Octree:
    def __init__(self, cell: CellMesh, levels: int):
        cen = cell.centroid
        lo, hi = cen.min(axis=0), cen.max(axis=0)
        self.c0 = 0.5 * (lo + hi)
        self.e0 = (hi - lo).max() * (1.0 + 1e-9)
        if not self.e0 > 0.0:
            self.e0 = 1.0          # all centroids at one point: one box at every level
        self.L = int(levels)
        self.corner = self.c0 - 0.5 * self.e0
        self.boxes = []          # per level: sorted list of occupied box keys (ix, iy, iz)
        self.elem_box = []       # per level: key of each element's box
        self.radius = []         # per level: largest centre-to-vertex distance of its boxes
        for l in range(self.L + 1):
            e = self.e0 / 2 ** l
            idx = np.floor((cen - self.corner) / e).astype(np.int64)
            idx = np.clip(idx, 0, 2 ** l - 1)
            keys = [tuple(v) for v in idx]
            self.elem_box.append(keys)
            self.boxes.append(sorted(set(keys), key=lambda t: (t[2], t[1], t[0])))
            ctr = self.corner[None, :] + (idx + 0.5) * e
            self.radius.append(float(np.linalg.norm(cell.v - ctr[:, None, :], axis=2).max()))

    def edge(self, l):
        return self.e0 / 2 ** l

    def centre(self, l, key):
        return self.corner + (np.asarray(key, dtype=np.float64) + 0.5) * self.edge(l)

    def children(self, l, key):
        out = []
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    c = (2 * key[0] + dx, 2 * key[1] + dy, 2 * key[2] + dz)
                    if c in self._occ(l + 1):
                        out.append(c)
        return out

    @lru_cache(maxsize=None)
    def _occ(self, l):
        return frozenset(self.boxes[l])

    def leaf_elements(self, key):
        return [j for j, k in enumerate(self.elem_box[self.L]) if k == key]


def interaction_lists(tree: Octree, shift):
    """(m2l, p2p) for one near offset: lists of (level, target key, source
    key) reached from the pair of roots."""
    m2l, p2p = [], []
    stack = [(0, (0, 0, 0), (0, 0, 0))]
    shift = np.asarray(shift, dtype=np.float64)
    while stack:
        l, a, b = stack.pop()
        d = tree.centre(l, a) - (tree.centre(l, b) + shift)
        if np.linalg.norm(d) >= 3.0 * tree.radius[l] * (1.0 - TIE):
            m2l.append((l, a, b))
        elif l == tree.L:
            p2p.append((a, b))
        else:
            for ca in tree.children(l, a):
                for cb in tree.children(l, b):
                    stack.append((l + 1, ca, cb))
    return m2l, p2p


def regular_translation(bvec, k, nt, rho=None, nq=None):
    """R (B x B) with I_q(a + b) = sum_q' R[q, q'] I_q'(a), by projection of
    I_q(rho u + b) on Y_q'(u) over the unit sphere (Gauss-Legendre in
    cos(theta), trapezoid in phi):  R[q, q'] = (2n'+1)/(4 pi j_n'(k rho)) *
    int I_q(rho u + b) conj(Y_q'(u)) dOmega."""
    coeffs = sp.coeff_list(nt)
    if rho is None:
        # the division by j_n'(k rho) amplifies quadrature rounding: take the
        # k rho in [1.5, 8] that keeps min_n |j_n(k rho)| largest
        grid = np.linspace(1.5, 8.0, 27)
        score = [min(abs(sp.sph_jn(n, x)) for n in range(nt + 1)) for x in grid]
        rho = grid[int(np.argmax(score))] / k
    if nq is None:
        nq = 2 * nt + 24 + int(k * np.linalg.norm(bvec))
    x, wx = np.polynomial.legendre.leggauss(nq)
    nphi = 2 * nq
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - x * x)
    U = np.stack([st[:, None] * np.cos(phi)[None], st[:, None] * np.sin(phi)[None],
                  x[:, None] * np.ones_like(phi)[None]], axis=-1).reshape(-1, 3)
    W = (wx[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).ravel()
    Iab = sp.wave_table(nt, rho * U + np.asarray(bvec, dtype=np.float64)[None], k, "I")
    Y = sp.sph_harm_table(nt, U)
    jn = np.array([sp.sph_jn(n, k * rho) for n, m in coeffs])
    f2 = np.array([2 * n + 1 for n, m in coeffs], dtype=np.float64)
    return (Iab * W[None]) @ np.conj(Y).T * f2[None, :] / (4 * np.pi * jn[None, :])


@lru_cache(maxsize=None)
def _regular_translation_cached(b, k, nt):
    return regular_translation(np.array(b), k, nt)


def m2m_matrix(child_c, parent_c, k, nt):
    """M(c_p) = T M(c_c),  T = conj(R(c_c - c_p))."""
    b = tuple(float(v) for v in np.asarray(child_c) - np.asarray(parent_c))
    return np.conj(_regular_translation_cached(b, float(k), int(nt)))


def l2l_matrix(parent_c, child_c, k, nt):
    """L(c_c) = T L(c_p),  T[q', q] = (2n+1)/(2n'+1) conj(R[q, q'](c_c - c_p))."""
    b = tuple(float(v) for v in np.asarray(child_c) - np.asarray(parent_c))
    R = _regular_translation_cached(b, float(k), int(nt))
    f = np.array([2 * n + 1 for n, m in sp.coeff_list(nt)], dtype=np.float64)
    return (np.conj(R) * f[:, None] / f[None, :]).T


def p2m_leaf(cell: CellMesh, elems, centre, k, nt, beta=0.0):
    """V (B x len(elems)) about the leaf centre, as fmm.p2m_table."""
    v = cell.v[elems]
    pts, w = collapsed_rule(v[:, 0], v[:, 1], v[:, 2], Q_FAR)
    rel = pts - np.asarray(centre)[None, None, :]
    g = sp.grad_regular_table(nt, rel, k)
    dIdn = np.einsum("bnqi,ni->bnq", g, cell.normal[elems])
    V = np.sum(np.conj(dIdn) * w[None], axis=2)
    if beta != 0:
        I = sp.wave_table(nt, rel.reshape(-1, 3), k, "I").reshape(-1, rel.shape[0], rel.shape[1])
        V = V + 1j * k * beta * np.sum(np.conj(I) * w[None], axis=2)
    return V


def l2p_leaf(cell: CellMesh, elems, centre, k, nt):
    """U (len(elems) x B) about the leaf centre, as fmm.l2p_table."""
    x = cell.centroid[elems] - np.asarray(centre)[None, :]
    I = sp.wave_table(nt, x, k, "I")
    g = sp.grad_regular_table(nt, x, k)
    dIdn = np.einsum("bni,ni->bn", g, cell.normal[elems])
    fac = np.array([-(1j * k / (4 * np.pi)) * (2 * n + 1) for n, m in sp.coeff_list(nt)])
    return (fac[:, None] * (np.conj(I) + coupling(k) * np.conj(dIdn))).T


def near_block_apply(cell: CellMesh, tree: Octree, shift, k, nt_near, x, S_exact, beta=0.0, p2m=None, l2p=None,
                     dofs=None):
    """S~_delta x for one near offset, x (R, n): P2M at the leaves of the
    source cell, M2M up the tree, M2L on the interaction list, L2L down, L2P
    at the leaves of the target cell, plus the P2P pairs taken from the exact
    block S_exact (n x n).  p2m, l2p: the leaf tables of the element family
    (default: flat triangles, p2m_leaf and l2p_leaf); dofs: the dof indices of
    a list of elements (default: one dof per element, the element's index)."""
    p2m = p2m_leaf if p2m is None else p2m
    l2p = l2p_leaf if l2p is None else l2p
    dofs = (lambda el: el) if dofs is None else dofs
    from .fmm import m2l_block
    x = np.atleast_2d(x)
    L = tree.L
    m2l, p2p = interaction_lists(tree, shift)
    Mom = [dict() for _ in range(L + 1)]
    for key in tree.boxes[L]:
        el = tree.leaf_elements(key)
        Mom[L][key] = x[:, dofs(el)] @ p2m(cell, el, tree.centre(L, key), k, nt_near, beta).T
    for l in range(L - 1, -1, -1):
        for key in tree.boxes[l]:
            acc = 0.0
            for ch in tree.children(l, key):
                acc = acc + Mom[l + 1][ch] @ m2m_matrix(tree.centre(l + 1, ch), tree.centre(l, key), k, nt_near).T
            Mom[l][key] = acc
    Loc = [dict() for _ in range(L + 1)]
    for l, a, b in m2l:
        K = m2l_block(tree.centre(l, a) - tree.centre(l, b) - np.asarray(shift), k, nt_near)
        Loc[l][a] = Loc[l].get(a, 0.0) + Mom[l][b] @ K.T
    for l in range(L):
        for key, val in Loc[l].items():
            for ch in tree.children(l, key):
                T = l2l_matrix(tree.centre(l, key), tree.centre(l + 1, ch), k, nt_near)
                Loc[l + 1][ch] = Loc[l + 1].get(ch, 0.0) + val @ T.T
    y = np.zeros((x.shape[0], x.shape[1]), dtype=complex)
    for key, val in Loc[L].items():
        el = tree.leaf_elements(key)
        y[:, dofs(el)] += val @ l2p(cell, el, tree.centre(L, key), k, nt_near).T
    for a, b in p2p:
        ia, jb = dofs(tree.leaf_elements(a)), dofs(tree.leaf_elements(b))
        y[:, ia] += x[:, jb] @ S_exact[np.ix_(ia, jb)].T
    return y


def near_block_matrix(cell: CellMesh, tree: Octree, lattice, delta, k, nt_near, beta=0.0, S_exact=None):
    """The matrix of S~_delta (n x n)."""
    if S_exact is None:
        S_exact = toeplitz_block(cell, lattice, delta, k, beta)
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    return near_block_apply(cell, tree, shift, k, nt_near, np.eye(cell.n), S_exact, beta).T


def fmm2_matvec_explicit(cell: CellMesh, lattice, counts, k, nt, nt_near, levels, p, beta=0.0):
    """Explicit FMPBEM2 product: the single-level FMPBEM of fmm.py with every
    near block S_delta replaced by its multilevel approximation."""
    from .fmm import fmm_matvec_explicit
    tree = Octree(cell, levels)
    near = {d: near_block_matrix(cell, tree, lattice, d, k, nt_near, beta) for d in near_offsets(counts)}
    return fmm_matvec_explicit(cell, lattice, counts, k, nt, p, near_blocks=near, beta=beta)

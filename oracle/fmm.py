"""Single-level fast multipole operators of the FMPBEM (Sec. 3.1-3.2,
Appendix A).  Oracle code: test infrastructure only.

Boxes are the unit cells (Sec. 3.2); the expansion centre of every cell is
its mesh origin.  With mesh normals (see ``oracle.bem``) the far part of the
collocation operator, -(D + b H) restricted to well-separated cells, is
approximated by
    y_i = sum_q U_0[i, q] L_q,
    L   = K(d) M,   d = x_c - y_c  (Eq. (m2l)),
    M_q = sum_j V_0[q, j] p_j      (Eq. (p2m)),
with
    V_0[q, j] = int_{E_j} dconj(I_q)(y - y_c)/dn_m(y) dA            (P2M),
    U_0[i, q] = -(ik/4pi)(2n+1) [conj(I_q)(x_i - x_c)
                 + b dconj(I_q)(x_i - x_c)/dn_m(x)]                   (L2P),
    K(d)[q, q'] = (2n'+1) (-1)^{m+m'} sum_{l in N} W_{n',n,m',m,l}
                 O_l^{m+m'}(d),
    W = (2l+1) i^{n-n'+l} (n n' l; 0 0 0) (n n' l; m m' -m-m')       (Eq. (wigner)),
q = n(n+1)+m.  Readings of garbled or silent points:
  * The phase of W is read as i^{n-n'+l}; the printed i^{n'-n+l} is the same
    formula with O_l evaluated at y_c - x_c (O_l(-d) = (-1)^l O_l(d) and
    l = n+n' mod 2).  Only this reading agrees with the independent
    projection M2L below and reproduces G.
  * N is taken as max(|m+m'|, |n-n'|) <= l <= n+n' with n+n'-l even; the
    printed strict inequalities drop the end terms and break the expansion.
  * The P2M integral uses the far-field rule of ``oracle.bem`` (q = 3
    collapsed Gauss-Legendre), so that U K V tends to the exact far blocks as
    the truncation number grows.
  * Near/far (Eq. (admissibility)) with r the cell edge: cells are near when
    the integer offset has max-norm <= 1 (the 3^d unique near blocks that the
    paper counts for square cells, Sec. 3.3).
"""
from functools import lru_cache

import numpy as np

from . import special as sp
from .bem import CellMesh, collapsed_rule, Q_FAR, coupling, toeplitz_block, lattice_cells


def far_rule_points(cell: CellMesh):
    """Far-field rule on every element: points (n, 9, 3), weights (n, 9)."""
    v = cell.v
    return collapsed_rule(v[:, 0], v[:, 1], v[:, 2], Q_FAR)


def p2m_table(cell: CellMesh, k: float, nt: int, beta=0.0):
    """V_0 (B x n): moments of each element's unit density (Eq. (p2m)).  With
    a uniform admittance beta the single-layer source term of Eq. (bm),
    i k beta int G dA, adds i k beta int conj(I_q)(y - y_c) dA (the target
    side, U_0, is the same operator 1 + b d/dn_x for both layers)."""
    pts, w = far_rule_points(cell)
    g = sp.grad_regular_table(nt, pts, k)               # B x n x 9 x 3
    dIdn = np.einsum("bnqi,ni->bnq", g, cell.normal)    # d I / dn_m
    V = np.sum(np.conj(dIdn) * w[None], axis=2)          # conj(dI/dn) = d conj(I)/dn
    if beta != 0:
        n9 = pts.shape[0] * pts.shape[1]
        I = sp.wave_table(nt, pts.reshape(n9, 3), k, "I").reshape(-1, pts.shape[0], pts.shape[1])
        V = V + 1j * k * beta * np.sum(np.conj(I) * w[None], axis=2)
    return V


def l2p_table(cell: CellMesh, k: float, nt: int):
    """U_0 (n x B): local expansion evaluated at the collocation points
    (Eq. (l2p) and its normal derivative), times -(ik/4pi)(2n+1)."""
    x = cell.centroid
    I = sp.wave_table(nt, x, k, "I")                    # B x n
    g = sp.grad_regular_table(nt, x, k)                  # B x n x 3
    dIdn = np.einsum("bni,ni->bn", g, cell.normal)
    b = coupling(k)
    fac = np.array([-(1j * k / (4 * np.pi)) * (2 * n + 1) for n, m in sp.coeff_list(nt)])
    return (fac[:, None] * (np.conj(I) + b * np.conj(dIdn))).T


@lru_cache(maxsize=None)
def _m2l_terms(nt: int):
    """Every nonzero term of Eq. (m2l): for entry (q, q') and l in N the
    coefficient (2n'+1)(-1)^{m+m'} W_{n',n,m',m,l} and the index of
    O_l^{m+m'}.  Returned as flat arrays (entry, O index, coefficient)."""
    coeffs = sp.coeff_list(nt)
    B = len(coeffs)
    ent, oidx, coef = [], [], []
    for qi, (n, m) in enumerate(coeffs):
        for qj, (n2, m2) in enumerate(coeffs):
            mu = m + m2
            for l in range(max(abs(mu), abs(n - n2)), n + n2 + 1):
                if (n + n2 - l) % 2:
                    continue
                w3 = sp.wigner3j(n, n2, l, 0, 0, 0) * sp.wigner3j(n, n2, l, m, m2, -mu)
                if w3 == 0.0:
                    continue
                W = (2 * l + 1) * (1j) ** ((n - n2 + l) % 4) * w3
                ent.append(qi * B + qj)
                oidx.append(sp.coeff_index(l, mu))
                coef.append((2 * n2 + 1) * (-1) ** ((m + m2) % 2) * W)
    return np.array(ent), np.array(oidx), np.array(coef)


def m2l_block(dvec, k: float, nt: int):
    """K(d) (B x B) from Eqs. (m2l), (wigner) with O_l evaluated at d."""
    O = sp.wave_table(2 * nt, np.asarray(dvec, dtype=np.float64), k, "O")
    ent, oidx, coef = _m2l_terms(nt)
    B = (nt + 1) ** 2
    K = np.zeros(B * B, dtype=complex)
    np.add.at(K, ent, coef * O[oidx])
    return K.reshape(B, B)


def m2l_block_by_projection(dvec, k: float, nt: int, rho0: float, nq: int = 48):
    """Independent M2L: K[q, q'] = (2n'+1)/(4 pi j_n(k rho0)) *
    int_{|u|=1} O_{n'}^{m'}(d + rho0 u) Y_n^m(u) dOmega(u), by Gauss-Legendre
    in cos(theta) times the trapezoid rule in phi.  Derived from the
    orthogonality of Y_n^m (int |Y_n^m|^2 = 4 pi/(2n+1)) applied to the local
    expansion of Eq. (l2p); needs rho0 < |d| and j_n(k rho0) != 0."""
    x, wx = np.polynomial.legendre.leggauss(nq)
    nphi = 2 * nq
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - x * x)
    U = np.stack([st[:, None] * np.cos(phi)[None], st[:, None] * np.sin(phi)[None],
                  x[:, None] * np.ones_like(phi)[None]], axis=-1).reshape(-1, 3)
    W = (wx[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).ravel()
    O = sp.wave_table(nt, np.asarray(dvec)[None, :] + rho0 * U, k, "O")     # B x Q
    Y = sp.wave_table(nt, U, 1.0, "I") / np.array(
        [sp.sph_jn(n, 1.0) for n, m in sp.coeff_list(nt)])[:, None]        # Y_n^m(u)
    coeffs = sp.coeff_list(nt)
    jn = np.array([sp.sph_jn(n, k * rho0) for n, m in coeffs])
    proj = (Y * W[None]) @ O.T                                              # [q, q']
    fac2 = np.array([2 * n2 + 1 for n2, m2 in coeffs])
    return proj * fac2[None, :] / (4 * np.pi * jn[:, None])


def fmm_matvec_explicit(cell: CellMesh, lattice, counts, k, nt, p, near_blocks=None,
                        V0=None, U0=None, beta=0.0):
    """Explicit, unconvolved FMPBEM product (Eq. (2dPeriodicFMM)):
    y_c = sum_{near c'} S_{c-c'} p_{c'} + U_0 sum_{far c'} K((c-c').a) V_0 p_{c'},
    looping over every cell pair -- no FFT, no circulant embedding."""
    p = np.atleast_2d(p)
    L = np.asarray(lattice, dtype=np.float64)
    cells = lattice_cells(counts)
    n = cell.n
    R = p.shape[0]
    P = p.reshape(R, len(cells), n)
    if near_blocks is None:
        near_blocks = {}
    V0 = p2m_table(cell, k, nt, beta) if V0 is None else V0
    U0 = l2p_table(cell, k, nt) if U0 is None else U0
    Mom = P @ V0.T                                       # R x Nc x B
    Y = np.zeros((R, len(cells), n), dtype=complex)
    Kcache = {}
    for ci, c in enumerate(cells):
        Lc = np.zeros((R, V0.shape[0]), dtype=complex)
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(c, cp))
            if max(abs(x) for x in delta) <= 1:
                if delta not in near_blocks:
                    near_blocks[delta] = toeplitz_block(cell, L, delta, k, beta)
                Y[:, ci] += P[:, cj] @ near_blocks[delta].T
            else:
                if delta not in Kcache:
                    Kcache[delta] = m2l_block(np.asarray(delta, dtype=np.float64) @ L, k, nt)
                Lc += Mom[:, cj] @ Kcache[delta].T
        Y[:, ci] += Lc @ U0.T
    return Y.reshape(R, -1)


# ------------------------------------------------------ truncation rule --
# The paper asks for a truncation number that is "sufficiently large"
# (Sec. 3.1) and shows that the needed n_t grows with frequency (Sec. 4,
# the accuracy study: n_t = 4 enough at 100 Hz, n_t >= 6 at 1 kHz).  The
# rule read from that: the smallest n_t >= 4 for which the multipole form
# U_0 K(d) V_0 of the block of the nearest far cell reproduces the exact
# block T_d on a fixed set of probe vectors to a relative 1e-6.

def probe_vectors(n, count=4):
    """The probe vectors of the truncation rule, rows p < count:
    x_j = exp(2 pi i frac((p + 1) j phi)), phi = (sqrt(5) - 1) / 2, j < n
    (a deterministic, well-spread sequence; no random draw)."""
    phi = (np.sqrt(5.0) - 1.0) / 2.0
    j = np.arange(n, dtype=np.float64)
    out = np.empty((count, n), dtype=complex)
    for p in range(count):
        t = np.fmod((p + 1) * j * phi, 1.0)
        out[p] = np.exp(2j * np.pi * t)
    return out


def nearest_far_offset(lattice, counts):
    """The far offset (max-norm >= 2, inside the grid's offset range) whose
    translation d . lattice is shortest; ties go to the first in the order
    dz, dy, dx ascending.  None if the grid has no far cell pair."""
    L = np.asarray(lattice, dtype=np.float64)
    M = list(counts) + [1] * (3 - len(counts))
    best, bd = None, np.inf
    for dz in range(1 - M[2], M[2]):
        for dy in range(1 - M[1], M[1]):
            for dx in range(1 - M[0], M[0]):
                if max(abs(dx), abs(dy), abs(dz)) <= 1:
                    continue
                d = np.linalg.norm(np.array([dx, dy, dz], dtype=np.float64) @ L)
                if d < bd:
                    best, bd = (dx, dy, dz), d
    return best


def truncation_errors(cell: CellMesh, lattice, counts, k, beta=0.0, nt_min=4, nt_max=20, block=None):
    """{n_t: ||(U_0 K(d) V_0 - T_d) X|| / ||T_d X||} over n_t_min..n_t_max for
    the nearest far offset d and the probe vectors X (Frobenius norms over
    the probes).  The tables of n_t are the leading (n_t + 1)^2 rows and
    columns of those of n_t_max (every entry depends only on its degrees and
    orders).  block: T_d if already computed."""
    d = nearest_far_offset(lattice, counts)
    if d is None:
        return None, {}
    L = np.asarray(lattice, dtype=np.float64)
    T = toeplitz_block(cell, L, d, k, beta) if block is None else block
    X = probe_vectors(cell.n)
    TX = X @ T.T
    V = p2m_table(cell, k, nt_max, beta)
    U = l2p_table(cell, k, nt_max)
    K = m2l_block(np.asarray(d, dtype=np.float64) @ L, k, nt_max)
    errs = {}
    for nt in range(nt_min, nt_max + 1):
        B = (nt + 1) ** 2
        Y = ((X @ V[:B].T) @ K[:B, :B].T) @ U[:, :B].T
        errs[nt] = np.linalg.norm(Y - TX) / np.linalg.norm(TX)
    return d, errs


def auto_truncation(cell: CellMesh, lattice, counts, k, beta=0.0, tol=1e-6, nt_min=4, nt_max=20):
    """The truncation rule: the smallest n_t in nt_min..nt_max meeting tol
    (nt_min when the grid has no far cell pair; None when no n_t up to
    nt_max meets it)."""
    d, errs = truncation_errors(cell, lattice, counts, k, beta, nt_min, nt_max)
    if d is None:
        return nt_min
    for nt in range(nt_min, nt_max + 1):
        if errs[nt] <= tol:
            return nt
    return None

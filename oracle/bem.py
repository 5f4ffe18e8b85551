"""Burton-Miller collocation BEM (Sec. 2.1), constant flat-triangle elements,
for a rigid boundary or a uniform admittance, and its multilevel block
Toeplitz form for finite periodic arrays (Sec. 2.2).  Oracle code: test
infrastructure only.

Equation solved (Eq. (bm) with Eq. (admittance); beta = 0 is the rigid case).
The paper's normal points out of the fluid (that is the orientation under
which its CBIE, Eq. (cbie), follows from Green's identity and gives
c = 1/2 for p = p_inc = 1 at k -> 0).  Meshes here carry normals n_m into the
fluid, n_m = -n, so in mesh normals the collocation equation at centroid x_i
reads
    1/2 p_i - sum_j [D_ij + b H_ij] p_j = p_inc(x_i) + b dp_inc/dn_m(x_i),
    D_ij = int_{E_j} dG/dn_m(y) dA_y,   H_ij = int_{E_j} d2G/dn_m(x)dn_m(y) dA_y,
    b = -alpha = i/k   (alpha = -i/k, the coupling of Eq. (bm)),
with G = e^{ikr}/(4 pi r) (Eq. (green3dFull)).  The matrix entry is
A_ij = 1/2 delta_ij - (D_ij + b H_ij).

Admittance (Eq. (admittance)): dp/dn = i k beta p with the paper's normal n,
i.e. dp/dn_m = -i k beta p in mesh normals.  The dp/dn terms of Eq. (bm),
(alpha/2) dp/dn(x) - int [G + alpha dG/dn(x)] dp/dn dA, then add
    A_ij += (beta/2) delta_ij - i k beta (S_ij + b K_ij),
    S_ij = int_{E_j} G dA_y,   K_ij = int_{E_j} dG/dn_m(x) dA_y,
(alpha i k beta / 2 = beta / 2 and alpha dG/dn = b dG/dn_m), the matrix
H - G Y of Eq. (matrixBEM) with a uniform normalised admittance beta.

Quadrature (the paper names the element type only, Eq. (matrixBEM)); the
rule below is part of the operator's definition and the GPU library
generates the same rule from the same description:
  * collapsed Gauss-Legendre rule of order q on a triangle (a, b, c) with apex
    a: y(s,t) = a + s[(b-a) + t(c-b)], dA = 2 area s ds dt, q x q nodes;
  * d = |x_i - centroid_j|, h_j = longest edge of E_j, thresholds scaled by
    (1 + 1e-9) so that exact ties go to the more accurate class:
      far        d >= 4 h_j          : q = 3 on E_j (apex v0)
      near       1.5 h_j <= d < 4 h_j: q = 8 on E_j
      very near  d < 1.5 h_j, j != i : q = 8 on each of the four midpoint
                 children (v0,m01,m20), (m01,v1,m12), (m20,m12,v2), (m01,m12,m20)
      self       j == i (x_i on E_i) : D = 0 (flat panel); H = finite part
                 (1/4pi)[ fp int r^-3 dA  +  int (e^{ikr}(1-ikr) - 1) r^-3 dA ],
                 the first in closed form -sum_edges (t_b/|b-x| - t_a/|a-x|)/h_e,
                 the second on the three children (x, v_a, v_b) with apex x, q = 8;
                 S = (1/4pi)[ int r^-1 dA + int (e^{ikr} - 1) r^-1 dA ], the first in
                 closed form sum_edges h_e ln((t_b + |b-x|)/(t_a + |a-x|)), the second
                 on the same three children; K = 0 (flat panel).
"""
import numpy as np

FAR_RATIO = 4.0
NEAR_RATIO = 1.5
# ties (d/h within 1e-9 of a threshold, which regular meshes produce exactly)
# go to the more accurate class, so that rounding cannot flip a decision
TIE = 1e-9
Q_FAR = 3
Q_NEAR = 8
Q_SELF = 8


# ------------------------------------------------------------ geometry -----

class CellMesh:
    """Per-element geometry of one unit-cell mesh (target cell at the origin)."""

    def __init__(self, verts, tris):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        v = self.verts[self.tris]                       # n x 3 x 3
        self.v = v
        cr = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
        two_area = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * two_area
        self.normal = cr / two_area[:, None]
        self.centroid = v.mean(axis=1)
        edges = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 1], v[:, 0] - v[:, 2]], axis=1)
        self.hmax = np.linalg.norm(edges, axis=2).max(axis=1)
        self.n = len(self.tris)


def gauss_legendre_01(q: int):
    """Gauss-Legendre nodes and weights on [0, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def collapsed_rule(a, b, c, q: int):
    """Nodes (..., q*q, 3) and weights (..., q*q) of the collapsed rule with
    apex a on triangle(s) (a, b, c)."""
    t1, w1 = gauss_legendre_01(q)
    s = t1[:, None] * np.ones(q)[None, :]            # s index slow
    t = np.ones(q)[:, None] * t1[None, :]
    ws = (w1[:, None] * w1[None, :]).ravel()
    s, t = s.ravel(), t.ravel()
    a, b, c = (np.asarray(z)[..., None, :] for z in (a, b, c))
    pts = a + s[:, None] * ((b - a) + t[:, None] * (c - b))
    cr = np.cross(b[..., 0, :] - a[..., 0, :], c[..., 0, :] - a[..., 0, :])
    two_area = np.linalg.norm(cr, axis=-1)
    w = two_area[..., None] * s * ws
    return pts, w


def element_rule(tri_v, cls: str):
    """Rule for whole elements tri_v (..., 3, 3) of class 'far' / 'near' /
    'verynear'."""
    v0, v1, v2 = tri_v[..., 0, :], tri_v[..., 1, :], tri_v[..., 2, :]
    if cls == "far":
        return collapsed_rule(v0, v1, v2, Q_FAR)
    if cls == "near":
        return collapsed_rule(v0, v1, v2, Q_NEAR)
    m01, m12, m20 = 0.5 * (v0 + v1), 0.5 * (v1 + v2), 0.5 * (v2 + v0)
    parts = [(v0, m01, m20), (m01, v1, m12), (m20, m12, v2), (m01, m12, m20)]
    P, W = zip(*[collapsed_rule(a, b, c, Q_NEAR) for a, b, c in parts])
    return np.concatenate(P, axis=-2), np.concatenate(W, axis=-1)


# ------------------------------------------------------------- kernels -----

def kernel_dlp(x, nx, y, ny, k):
    """dG/dn_y = e^{ikr}(1 - ikr) ((x-y).n_y) / (4 pi r^3)."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    e = np.exp(1j * k * r)
    return e * (1.0 - 1j * k * r) * np.einsum("...i,...i->...", d, ny) / (4 * np.pi * r ** 3)


def kernel_hyp(x, nx, y, ny, k):
    """d2G/dn_x dn_y = e^{ikr}[(1-ikr) r^2 (n_x.n_y) - (3 - 3ikr - k^2 r^2)
    ((x-y).n_x)((x-y).n_y)] / (4 pi r^5)."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    e = np.exp(1j * k * r)
    dnx = np.einsum("...i,...i->...", d, nx)
    dny = np.einsum("...i,...i->...", d, ny)
    nn = np.einsum("...i,...i->...", nx * np.ones_like(d), ny * np.ones_like(d))
    ikr = 1j * k * r
    return e * ((1.0 - ikr) * r * r * nn - (3.0 - 3.0 * ikr - (k * r) ** 2) * dnx * dny) / (4 * np.pi * r ** 5)


def kernel_slp(x, y, k):
    """G = e^{ikr} / (4 pi r)."""
    r = np.linalg.norm(x - y, axis=-1)
    return np.exp(1j * k * r) / (4 * np.pi * r)


def kernel_adlp(x, nx, y, k):
    """dG/dn_x = e^{ikr}(ikr - 1) ((x-y).n_x) / (4 pi r^3)."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    return np.exp(1j * k * r) * (1j * k * r - 1.0) * np.einsum("...i,...i->...", d, nx) / (4 * np.pi * r ** 3)


def _sin_minus_xcos(x):
    """sin x - x cos x without cancellation (series below 0.5)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.sin(x) - x * np.cos(x)
    small = np.abs(x) < 0.5
    if np.any(small):
        xs = x[small]
        acc = np.zeros_like(xs)
        term_fact = 1.0
        for j in range(1, 10):
            # (-1)^{j+1} 2j x^{2j+1} / (2j+1)!
            term_fact = 1.0
            for f in range(2, 2 * j + 2):
                term_fact *= f
            acc += (-1) ** (j + 1) * 2 * j * xs ** (2 * j + 1) / term_fact
        out[small] = acc
    return out


def self_hyp(tri_v, k):
    """Finite-part integral of d2G/dn_x dn_y over the flat element tri_v for x
    at its centroid (Hadamard finite part of the r^-3 term in closed form,
    the weakly singular remainder by polar quadrature)."""
    x = tri_v.mean(axis=0)
    fp = 0.0
    for e in range(3):
        a, b = tri_v[e], tri_v[(e + 1) % 3]
        eh = (b - a) / np.linalg.norm(b - a)
        ta, tb = np.dot(a - x, eh), np.dot(b - x, eh)
        he = np.linalg.norm((a - x) - ta * eh)
        fp -= (tb / np.linalg.norm(b - x) - ta / np.linalg.norm(a - x)) / he
    rem = 0.0 + 0.0j
    for e in range(3):
        a, b = tri_v[e], tri_v[(e + 1) % 3]
        pts, w = collapsed_rule(x, a, b, Q_SELF)
        r = np.linalg.norm(pts - x, axis=-1)
        kr = k * r
        re = -2.0 * np.sin(0.5 * kr) ** 2 + kr * np.sin(kr)      # cos kr + kr sin kr - 1
        im = _sin_minus_xcos(kr)                               # sin kr - kr cos kr
        rem += np.sum(w * (re + 1j * im) / r ** 3)
    return (fp + rem) / (4 * np.pi)


def inv_r_integral(tri_v, x):
    """Closed form of int_T 1/|x - y| dA_y for x in the plane of T and inside
    it: in polar coordinates about x the integral is int R(theta) dtheta, and
    each edge (foot of the perpendicular at distance h, coordinates t along
    the edge) gives h ln((t_b + |b - x|) / (t_a + |a - x|))."""
    total = 0.0
    for e in range(3):
        a, b = tri_v[e], tri_v[(e + 1) % 3]
        eh = (b - a) / np.linalg.norm(b - a)
        ta, tb = np.dot(a - x, eh), np.dot(b - x, eh)
        he = np.linalg.norm((a - x) - ta * eh)
        total += he * np.log((tb + np.linalg.norm(b - x)) / (ta + np.linalg.norm(a - x)))
    return total


def self_slp(tri_v, k):
    """Integral of G over the flat element tri_v for x at its centroid: the
    1/r part in closed form (polar coordinates about x: each edge contributes
    h ln((t_b + |b-x|)/(t_a + |a-x|))), the bounded remainder
    (e^{ikr} - 1)/r by polar quadrature on the three children (x, a, b)."""
    x = tri_v.mean(axis=0)
    closed = inv_r_integral(tri_v, x)
    rem = 0.0 + 0.0j
    for e in range(3):
        a, b = tri_v[e], tri_v[(e + 1) % 3]
        pts, w = collapsed_rule(x, a, b, Q_SELF)
        r = np.linalg.norm(pts - x, axis=-1)
        kr = k * r
        rem += np.sum(w * (-2.0 * np.sin(0.5 * kr) ** 2 + 1j * np.sin(kr)) / r)   # (e^{ikr} - 1)/r
    return (closed + rem) / (4 * np.pi)


# ----------------------------------------------------- operator entries -----

def classify(x, cen, hmax):
    d = np.linalg.norm(x - cen, axis=-1)
    cls = np.full(d.shape, 2, dtype=np.int8)          # very near
    cls[d >= NEAR_RATIO * (1.0 + TIE) * hmax] = 1    # near
    cls[d >= FAR_RATIO * (1.0 + TIE) * hmax] = 0     # far
    return cls


def pair_integrals(xs, nxs, tri_v, k, cls_code, with_sk=False):
    """D and H integrals (and S, K when with_sk) for pairs (xs[p], nxs[p]) x
    element tri_v[p] (all of one class), vectorised over pairs."""
    name = {0: "far", 1: "near", 2: "verynear"}[cls_code]
    pts, w = element_rule(tri_v, name)
    cr = np.cross(tri_v[:, 1] - tri_v[:, 0], tri_v[:, 2] - tri_v[:, 0])
    ny = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    X = xs[:, None, :]
    NX = nxs[:, None, :]
    NY = ny[:, None, :]
    D = np.sum(w * kernel_dlp(X, NX, pts, NY, k), axis=1)
    H = np.sum(w * kernel_hyp(X, NX, pts, NY, k), axis=1)
    if not with_sk:
        return D, H
    S = np.sum(w * kernel_slp(X, pts, k), axis=1)
    K = np.sum(w * kernel_adlp(X, NX, pts, k), axis=1)
    return D, H, S, K


def dh_block(tgt: CellMesh, src_v, k, self_pairs=None, chunk=200000, with_sk=False):
    """D and H matrices (n_t x n_s) for collocation points of ``tgt`` and source
    elements with vertex coordinates ``src_v`` (n_s x 3 x 3, already placed),
    and S, K as well when with_sk.
    ``self_pairs``: boolean n_t x n_s mask of pairs (i, j) with x_i on E_j."""
    nt_, ns = tgt.n, len(src_v)
    cen = src_v.mean(axis=1)
    cr = np.cross(src_v[:, 1] - src_v[:, 0], src_v[:, 2] - src_v[:, 0])
    edges = np.stack([src_v[:, 1] - src_v[:, 0], src_v[:, 2] - src_v[:, 1], src_v[:, 0] - src_v[:, 2]], axis=1)
    hmax = np.linalg.norm(edges, axis=2).max(axis=1)
    cls = classify(tgt.centroid[:, None, :], cen[None, :, :], hmax[None, :])
    if self_pairs is not None:
        cls[self_pairs] = 3
    D = np.zeros((nt_, ns), dtype=complex)
    H = np.zeros((nt_, ns), dtype=complex)
    S = np.zeros((nt_, ns), dtype=complex)
    K = np.zeros((nt_, ns), dtype=complex)
    for c in (0, 1, 2):
        ii, jj = np.nonzero(cls == c)
        for s in range(0, len(ii), chunk):
            i, j = ii[s:s + chunk], jj[s:s + chunk]
            out = pair_integrals(tgt.centroid[i], tgt.normal[i], src_v[j], k, c, with_sk)
            D[i, j] = out[0]
            H[i, j] = out[1]
            if with_sk:
                S[i, j] = out[2]
                K[i, j] = out[3]
    ii, jj = np.nonzero(cls == 3)
    for i, j in zip(ii, jj):
        H[i, j] = self_hyp(src_v[j], k)
        if with_sk:
            S[i, j] = self_slp(src_v[j], k)          # K = 0 on the flat panel
    if with_sk:
        return D, H, S, K
    return D, H


def coupling(k):
    """b = i/k (mesh-normal form of alpha = -i/k, Eq. (bm))."""
    return 1j / k


def _entries(D, H, S, K, k, beta):
    """-(D + b H) - i k beta (S + b K) (without the diagonal terms)."""
    b = coupling(k)
    T = -(D + b * H)
    if beta != 0:
        T = T - 1j * k * beta * (S + b * K)
    return T


def toeplitz_block(cell: CellMesh, lattice, delta, k, beta=0.0):
    """T_delta (Eq. (blockToeplizMatrix), Sec. 2.2): target cell at the origin,
    source cell displaced by -delta . lattice.  Entry (i, j) is the matrix
    entry of collocation point i against element j; beta = uniform
    normalised admittance (0: rigid)."""
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    src_v = cell.v + shift[None, None, :]
    selfp = np.eye(cell.n, dtype=bool) if not np.any(delta) else None
    if beta == 0:
        D, H = dh_block(cell, src_v, k, self_pairs=selfp)
        S = K = None
    else:
        D, H, S, K = dh_block(cell, src_v, k, self_pairs=selfp, with_sk=True)
    T = _entries(D, H, S, K, k, beta)
    if selfp is not None:
        T += (0.5 + 0.5 * beta) * np.eye(cell.n)
    return T


def lattice_cells(counts):
    """Cell multi-indices (ix, iy, iz) in the order c = (iz*My + iy)*Mx + ix."""
    Mx, My, Mz = counts
    return [(ix, iy, iz) for iz in range(Mz) for iy in range(My) for ix in range(Mx)]


def assemble_full_mesh(verts, tris, lattice, counts):
    """All cells' elements as one mesh, element index c*n + e."""
    L = np.asarray(lattice, dtype=np.float64)
    nv = len(verts)
    V, T = [], []
    for ci, c in enumerate(lattice_cells(counts)):
        V.append(np.asarray(verts) + np.asarray(c, dtype=np.float64) @ L)
        T.append(np.asarray(tris) + ci * nv)
    return np.concatenate(V), np.concatenate(T)


def dense_matrix(verts, tris, lattice, counts, k, beta=0.0):
    """The conventional dense BM collocation matrix (Eq. (matrixBEM)) of the
    whole array, assembled pair by pair over the full mesh with no use of the
    periodic structure; beta = uniform normalised admittance (0: rigid)."""
    V, T = assemble_full_mesh(verts, tris, lattice, counts)
    m = CellMesh(V, T)
    if beta == 0:
        D, H = dh_block(m, m.v, k, self_pairs=np.eye(m.n, dtype=bool))
        S = K = None
    else:
        D, H, S, K = dh_block(m, m.v, k, self_pairs=np.eye(m.n, dtype=bool), with_sk=True)
    return (0.5 + 0.5 * beta) * np.eye(m.n) + _entries(D, H, S, K, k, beta)


def all_offsets(counts):
    Mx, My, Mz = counts
    return [(dx, dy, dz) for dz in range(1 - Mz, Mz) for dy in range(1 - My, My) for dx in range(1 - Mx, Mx)]


def near_offsets(counts):
    return [d for d in all_offsets(counts) if max(abs(x) for x in d) <= 1]


def toeplitz_matvec(blocks, counts, p):
    """Explicit multilevel block-Toeplitz product (Eq. (toeplitzBEM)):
    y_c = sum_{c'} T_{c-c'} p_{c'}, summing only the offsets present in
    ``blocks`` (a dict delta -> n x n).  p: (R, Nc*n) or (Nc*n,)."""
    p = np.atleast_2d(p)
    cells = lattice_cells(counts)
    n = next(iter(blocks.values())).shape[0]
    R = p.shape[0]
    P = p.reshape(R, len(cells), n)
    Y = np.zeros_like(P, dtype=complex)
    for ci, c in enumerate(cells):
        for cj, cp in enumerate(cells):
            delta = tuple(a - b for a, b in zip(c, cp))
            if delta in blocks:
                Y[:, ci] += P[:, cj] @ blocks[delta].T
    return Y.reshape(R, -1)


# ---------------------------------------------------------- right-hand side --

def plane_wave_rhs(cell: CellMesh, lattice, counts, k, direction, amp=1.0):
    """b_i = p_inc(x_i) + b dp_inc/dn_m(x_i) for p_inc = amp e^{ik d.x}
    (Eq. (planewave), Eq. (bm) right-hand side)."""
    L = np.asarray(lattice, dtype=np.float64)
    dvec = np.asarray(direction, dtype=np.float64)
    out = []
    for c in lattice_cells(counts):
        x = cell.centroid + np.asarray(c, dtype=np.float64) @ L
        pinc = amp * np.exp(1j * k * (x @ dvec))
        dpdn = 1j * k * (cell.normal @ dvec) * pinc
        out.append(pinc + coupling(k) * dpdn)
    return np.concatenate(out)


def field_points(verts, tris, lattice, counts, k, p, points, direction, amp=1.0, beta=0.0):
    """Total pressure in the fluid (Eq. (cbie) with c = 1):
    p(x) = p_inc(x) + sum_j D(x, E_j) p_j  (mesh normals).  With a uniform
    admittance the single-layer term -G dp/dn_m of Eq. (cbie), with
    dp/dn_m = -i k beta p (Eq. (admittance)), adds i k beta S(x, E_j) p_j."""
    V, T = assemble_full_mesh(verts, tris, lattice, counts)
    m = CellMesh(V, T)
    pts = np.asarray(points, dtype=np.float64)
    cls = classify(pts[:, None, :], m.centroid[None], m.hmax[None])
    out = amp * np.exp(1j * k * (pts @ np.asarray(direction, dtype=np.float64)))
    out = out.astype(complex)
    dummy_n = np.zeros_like(pts)
    for c in (0, 1, 2):
        ii, jj = np.nonzero(cls == c)
        if len(ii) == 0:
            continue
        nz = dummy_n[ii] + np.array([0, 0, 1.0])
        if beta == 0:
            d, _ = pair_integrals(pts[ii], nz, m.v[jj], k, c)
        else:
            d, _, sl, _ = pair_integrals(pts[ii], nz, m.v[jj], k, c, with_sk=True)
            d = d + 1j * k * beta * sl
        np.add.at(out, ii, d * p[jj])
    return out

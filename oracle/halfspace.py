"""Half-space problems (Sec. 2.3 and Sec. 3.4): the Burton-Miller operator with
the half-space Green's function of Eq. (green3dHalf),
    G_h(x, y) = G(x, y) + R_p G(x, y^),
y^ the mirror image of y in the plane that divides the two half-spaces, and its
split into a block Toeplitz part T (the full-space operator, bem.py) and an
image part T^ (Eq. (toeplitzBEMsymmetry)).  Oracle code: test infrastructure
only.

Plane and mirror.  The plane is {x : x[axis] = offset}; the mirror is
M(v) = v with v[axis] -> 2 offset - v[axis], i.e. M(v) = R v + 2 offset e
with the linear reflection R (v[axis] -> -v[axis]) and e the unit vector of
the axis.  The scatterers lie on one side of the plane (the fluid side).

Image element.  The y^ integrals over element E_j are integrals over the
mirrored element, whose normal is R n_j (the derivative of G(x, M y) along
n_j at y is the derivative of G(x, .) along R n_j at M y).  The mirrored
element is taken with vertices (M v0, M v2, M v1): the reversed winding makes
the normal computed from the vertices equal to R n_j, and the collapsed rules
of bem.py (apex at the first vertex) are applied to it unchanged.  The image
entries are R_p times the entries of bem.py for this element, with no jump
term (a collocation point never lies on a mirrored element).

Lattice roles.  Each lattice axis with more than one cell is either parallel
to the plane (L_a[axis] = 0) or perpendicular to it (L_a a multiple of e).  A
perpendicular axis h makes T^ a multilevel block Hankel matrix
(Eq. (blockToeplizMatrixSymmetry)): with c~_h = M_h - 1 - c_h on the source
side (the permutation P that reverses the cells along h) the image block
depends only on delta~ = c - c~', so T^ P is block Toeplitz (Sec. 2.4) with
blocks T^(delta~) between the target cell at the origin and the mirrored
unit cell shifted by
    shift(delta~) = -sum_a delta~_a L_a - (M_h - 1) L_h + 2 offset e
(without a perpendicular axis P = identity and the (M_h - 1) L_h term drops).

FMM form (Eq. (2dPeriodicFMM_halfspace), Eq. (greenFMMhalfspace)).  The image
part is S^ + U K^ V^: U is the full-space L2P table, V^ the P2M table of the
reflected unit cell (vertices R v, reversed winding) about the origin, and
K^(delta~) the M2L block of the translation x_c - y^_c = -shift(delta~).  The
near set of the image part is read from Eq. (admissibilityMirror) with r the
longest lattice vector among the axes with more than one cell:
delta~ is near iff |x_c - y^_c| < 2 r (ties, within 1e-9, go to far, as the
equality is admissible in the printed criterion).

Incident fields.  A plane wave amp e^{i k d.x} or a monopole amp e^{ikr}/r
(r = |x - x_s|; amp is the pressure amplitude at 1 m), each with its image
R_p p_inc(M x), so that the incident field alone satisfies the plane's
condition (dp/dn = 0 at the plane for R_p = 1, p = 0 for R_p = -1).
"""
import numpy as np

from . import bem, fmm

TIE = 1e-9


class Plane:
    """Symmetry plane {x : x[axis] = offset} with reflection coefficient Rp."""

    def __init__(self, axis: int, offset: float, Rp: complex):
        self.axis = int(axis)
        self.offset = float(offset)
        self.Rp = complex(Rp)

    def e(self):
        v = np.zeros(3)
        v[self.axis] = 1.0
        return v

    def mirror(self, pts):
        """M(v) = v with v[axis] -> 2 offset - v[axis]."""
        p = np.array(pts, dtype=np.float64, copy=True)
        p[..., self.axis] = 2.0 * self.offset - p[..., self.axis]
        return p

    def reflect(self, vecs):
        """R v = v with v[axis] -> -v[axis] (the linear part of the mirror)."""
        v = np.array(vecs, dtype=np.float64, copy=True)
        v[..., self.axis] = -v[..., self.axis]
        return v


def image_tris(tris):
    """Reversed winding (v0, v2, v1) of the mirrored elements."""
    t = np.asarray(tris)
    return t[:, [0, 2, 1]]


def hankel_axis(lattice, counts, plane: Plane):
    """The lattice axis perpendicular to the plane (-1 if none); raises if an
    axis with more than one cell is neither parallel nor perpendicular."""
    L = np.asarray(lattice, dtype=np.float64)
    h = -1
    for a in range(3):
        if counts[a] <= 1:
            continue
        n = np.linalg.norm(L[a])
        along = abs(L[a][plane.axis])
        if along <= 1e-12 * n:
            continue
        if abs(along - n) <= 1e-12 * n:
            if h >= 0:
                raise ValueError("two lattice axes perpendicular to the plane")
            h = a
            continue
        raise ValueError(f"lattice vector {a} is neither parallel nor perpendicular to the plane")
    return h


def image_offsets(counts):
    """delta~ over the (2M-1)^d pattern, delta~_x fastest (as bem.all_offsets)."""
    return bem.all_offsets(counts)


def image_shift(lattice, counts, plane: Plane, dt):
    """shift(delta~) = -delta~ . L - (M_h - 1) L_h + 2 offset e."""
    L = np.asarray(lattice, dtype=np.float64)
    s = -np.asarray(dt, dtype=np.float64) @ L
    h = hankel_axis(lattice, counts, plane)
    if h >= 0:
        s = s - (counts[h] - 1) * L[h]
    return s + 2.0 * plane.offset * plane.e()


def reflected_cell(cell: bem.CellMesh, plane: Plane):
    """The unit cell reflected linearly (R v) with reversed winding: its
    element normals are R n_j and its expansion centre is the origin."""
    return bem.CellMesh(plane.reflect(cell.verts), image_tris(cell.tris))


def image_block(cell: bem.CellMesh, lattice, counts, plane: Plane, dt, k, beta=0.0):
    """T^(delta~): R_p times the entries of target cell at the origin against
    the reflected unit cell shifted by shift(delta~)."""
    rc = reflected_cell(cell, plane)
    src_v = rc.v + image_shift(lattice, counts, plane, dt)[None, None, :]
    if beta == 0:
        D, H = bem.dh_block(cell, src_v, k)
        S = K = None
    else:
        D, H, S, K = bem.dh_block(cell, src_v, k, with_sk=True)
    return plane.Rp * bem._entries(D, H, S, K, k, beta)


def reverse_cells(p, counts, h):
    """P p: cells reversed along axis h (identity for h < 0).  p: (R, Nc*n)."""
    p = np.atleast_2d(p)
    if h < 0:
        return p.copy()
    Mx, My, Mz = counts
    R = p.shape[0]
    n = p.shape[1] // (Mx * My * Mz)
    P = p.reshape(R, Mz, My, Mx, n)
    P = np.flip(P, axis={0: 3, 1: 2, 2: 1}[h])
    return np.ascontiguousarray(P).reshape(R, -1)


def dense_matrix_halfspace(verts, tris, lattice, counts, k, plane: Plane, beta=0.0):
    """The dense collocation matrix of the whole array with G_h, assembled pair
    by pair over the full mesh and its mirror image (Eq. (toeplitzBEMsymmetry)
    without any structure): A = A_full + R_p A^, A^_ij the entries of x_i
    against the mirrored element j (vertices (M v0, M v2, M v1))."""
    A = bem.dense_matrix(verts, tris, lattice, counts, k, beta)
    V, T = bem.assemble_full_mesh(verts, tris, lattice, counts)
    m = bem.CellMesh(V, T)
    img_v = plane.mirror(m.verts)[image_tris(m.tris)]
    if beta == 0:
        D, H = bem.dh_block(m, img_v, k)
        S = K = None
    else:
        D, H, S, K = bem.dh_block(m, img_v, k, with_sk=True)
    return A + plane.Rp * bem._entries(D, H, S, K, k, beta)


def structured_matvec_halfspace(cell: bem.CellMesh, lattice, counts, k, plane: Plane, p, beta=0.0,
                                blocks=None, image_blocks=None):
    """(T + T^) p as the two block Toeplitz products of Sec. 2.4: T p with the
    full-space blocks, and (T^ P)(P p) with the image blocks (Sec. 2.4, the
    Hankel part applied through the permutation P)."""
    p = np.atleast_2d(p)
    h = hankel_axis(lattice, counts, plane)
    if blocks is None:
        blocks = {d: bem.toeplitz_block(cell, lattice, d, k, beta) for d in bem.all_offsets(counts)}
    if image_blocks is None:
        image_blocks = {d: image_block(cell, lattice, counts, plane, d, k, beta) for d in image_offsets(counts)}
    y = bem.toeplitz_matvec(blocks, counts, p)
    y = y + bem.toeplitz_matvec(image_blocks, counts, reverse_cells(p, counts, h))
    return y


# ----------------------------------------------------------- incident field --

def _plane_wave(x, n, k, d, amp):
    ph = amp * np.exp(1j * k * (x @ d))
    return ph, 1j * k * (n @ d) * ph


def _monopole(x, n, k, xs, amp):
    r_vec = x - xs
    r = np.linalg.norm(r_vec, axis=-1)
    ph = amp * np.exp(1j * k * r) / r
    # d/dn (e^{ikr}/r) = e^{ikr} (ikr - 1)/r^2 * (r_vec . n)/r
    dn = ph * (1j * k * r - 1.0) / r * np.einsum("...i,...i->...", r_vec, n) / r
    return ph, dn


def incident(x, n, k, kind, vec, amp, plane: Plane = None):
    """p_inc and dp_inc/dn at points x with normals n; kind 'plane' (vec =
    unit direction) or 'monopole' (vec = source position), plus the image
    R_p p_inc(M x) when a plane is given."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    n = np.atleast_2d(np.asarray(n, dtype=np.float64))
    vec = np.asarray(vec, dtype=np.float64)
    f = _plane_wave if kind == "plane" else _monopole
    p, dp = f(x, n, k, vec, amp)
    if plane is not None and plane.Rp != 0:
        # p_inc(M x) has gradient R grad p_inc(M x): its normal derivative along
        # n is the derivative of p_inc at M x along R n
        pi, dpi = f(plane.mirror(x), plane.reflect(n), k, vec, amp)
        p = p + plane.Rp * pi
        dp = dp + plane.Rp * dpi
    return p, dp


def rhs(cell: bem.CellMesh, lattice, counts, k, kind, vec, amp=1.0, plane: Plane = None):
    """b_i = p_inc(x_i) + b dp_inc/dn_m(x_i) over every cell (Eq. (bm))."""
    L = np.asarray(lattice, dtype=np.float64)
    out = []
    for c in bem.lattice_cells(counts):
        x = cell.centroid + np.asarray(c, dtype=np.float64) @ L
        p, dp = incident(x, cell.normal, k, kind, vec, amp, plane)
        out.append(p + bem.coupling(k) * dp)
    return np.concatenate(out)


def field_points(verts, tris, lattice, counts, k, p, points, kind, vec, amp=1.0, plane: Plane = None, beta=0.0):
    """Total pressure in the fluid (Eq. (cbie) with c = 1 and G_h):
    p(x) = p_inc(x) + sum_j [D(x, E_j) + i k beta S(x, E_j)] p_j
           + R_p sum_j [D(x, E^_j) + i k beta S(x, E^_j)] p_j."""
    V, T = bem.assemble_full_mesh(verts, tris, lattice, counts)
    pts = np.asarray(points, dtype=np.float64)
    nz = np.zeros_like(pts) + np.array([0.0, 0.0, 1.0])
    out, _ = incident(pts, nz, k, kind, vec, amp, plane)
    out = out.astype(complex)
    meshes = [(bem.CellMesh(V, T), 1.0)]
    if plane is not None and plane.Rp != 0:
        meshes.append((bem.CellMesh(plane.mirror(V), image_tris(T)), plane.Rp))
    for m, scale in meshes:
        cls = bem.classify(pts[:, None, :], m.centroid[None], m.hmax[None])
        for c in (0, 1, 2):
            ii, jj = np.nonzero(cls == c)
            if len(ii) == 0:
                continue
            if beta == 0:
                d, _ = bem.pair_integrals(pts[ii], nz[ii], m.v[jj], k, c)
            else:
                d, _, sl, _ = bem.pair_integrals(pts[ii], nz[ii], m.v[jj], k, c, with_sk=True)
                d = d + 1j * k * beta * sl
            np.add.at(out, ii, scale * d * p[jj])
    return out


# ------------------------------------------------------------------ FMM form --

def image_r(lattice, counts):
    """r of Eq. (admissibilityMirror): the longest lattice vector among the
    axes with more than one cell."""
    L = np.asarray(lattice, dtype=np.float64)
    lens = [np.linalg.norm(L[a]) for a in range(3) if counts[a] > 1]
    return max(lens) if lens else np.linalg.norm(L, axis=1).max()


def image_near_offsets(lattice, counts, plane: Plane):
    """delta~ whose mirrored cell is not admissible: |x_c - y^_c| < 2 r."""
    r = image_r(lattice, counts)
    out = []
    for d in image_offsets(counts):
        t = -image_shift(lattice, counts, plane, d)
        if np.linalg.norm(t) < 2.0 * r * (1.0 - TIE):
            out.append(d)
    return out


def fmm_image_matvec_explicit(cell: bem.CellMesh, lattice, counts, k, nt, plane: Plane, p, beta=0.0):
    """The image part of Eq. (2dPeriodicFMM_halfspace), (S^ + U K^ V^) p, by
    explicit loops over every (target cell, mirrored source cell) pair:
    near pairs (Eq. (admissibilityMirror)) by the image blocks, far pairs by
    the expansion of Eq. (greenFMMhalfspace) about the mirrored centre."""
    p = np.atleast_2d(p)
    h = hankel_axis(lattice, counts, plane)
    q = reverse_cells(p, counts, h)
    cells = bem.lattice_cells(counts)
    n = cell.n
    R = p.shape[0]
    Q = q.reshape(R, len(cells), n)
    near = set(image_near_offsets(lattice, counts, plane))
    rc = reflected_cell(cell, plane)
    V0h = plane.Rp * fmm.p2m_table(rc, k, nt, beta)
    U0 = fmm.l2p_table(cell, k, nt)
    Mom = Q @ V0h.T
    Y = np.zeros((R, len(cells), n), dtype=complex)
    cache = {}
    for ci, c in enumerate(cells):
        Lc = np.zeros((R, V0h.shape[0]), dtype=complex)
        for cj, cq in enumerate(cells):
            dt = tuple(a - b for a, b in zip(c, cq))
            if dt in near:
                if dt not in cache:
                    cache[dt] = image_block(cell, lattice, counts, plane, dt, k, beta)
                Y[:, ci] += Q[:, cj] @ cache[dt].T
            else:
                key = ("K", dt)
                if key not in cache:
                    cache[key] = fmm.m2l_block(-image_shift(lattice, counts, plane, dt), k, nt)
                Lc += Mom[:, cj] @ cache[key].T
        Y[:, ci] += Lc @ U0.T
    return Y.reshape(R, -1)


# ----------------------------------------------------------- insertion loss --

def insertion_loss_from_fields(p_inc, p_tot):
    """Eq. (insertionloss): IL = 20 log10(sum_i |p_inc(x_i)| / sum_i |p(x_i)|)
    over the observation points, p_inc and p the fields of all sources
    together (arrays over the points)."""
    return 20.0 * np.log10(np.sum(np.abs(p_inc)) / np.sum(np.abs(p_tot)))


def insertion_loss(verts, tris, lattice, counts, k, P, points, incidents, plane: Plane = None, beta=0.0):
    """IL of the solutions P (R x N, one row per incident field of
    `incidents` = [(kind, vec, amp)]) at the observation points: the sources
    act together, so the fields of the R right-hand sides are summed."""
    pts = np.asarray(points, dtype=np.float64)
    nz = np.zeros_like(pts) + np.array([0.0, 0.0, 1.0])
    tot = np.zeros(len(pts), dtype=complex)
    inc = np.zeros(len(pts), dtype=complex)
    for r, (kind, vec, amp) in enumerate(incidents):
        tot += field_points(verts, tris, lattice, counts, k, P[r], pts, kind, vec, amp, plane, beta)
        inc += incident(pts, nz, k, kind, vec, amp, plane)[0]
    return insertion_loss_from_fields(inc, tot)

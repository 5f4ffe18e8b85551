"""Burton-Miller collocation on nine-node quadratic quadrilaterals (the
paper's element family, Sec. 2.1 and Eq. (matrixBEM), with the constant
discontinuous pressure of its first example): one pressure value per
element, collocated at the element centre.  Oracle code: test infrastructure
only.

Element.  y(xi, eta) = sum_a N_a(xi, eta) y_a on [-1, 1]^2 with N_a the
products of the 1-D quadratic Lagrange polynomials on the nodes -1, 0, 1
(node (i, j) at 3 j + i, i along xi).  Jacobian vector J = y_xi x y_eta,
normal n = J / |J| (into the fluid), dA = |J| dxi deta.  The collocation
point of element i is x_i = y(0, 0) with normal n_x = n(0, 0).

Integrals of element j seen from (x, n_x), with the kernels of bem.py
(dG/dn_y, d2G/dn_x dn_y, G, dG/dn_x):
  * regular (x not on element j), classes by d = |x - y_j(0, 0)| and the
    longest corner-to-corner chord h_j (thresholds as bem.py): far d >= 4 h:
    4 x 4 Gauss-Legendre; near 1.5 h <= d < 4 h: 8 x 8; very near: 8 x 8 on
    each of the four parameter quarters;
  * self (j = i): polar coordinates (rho, theta) about (0, 0) in the
    parameter plane, the square split into four triangles with apex at the
    centre, Gauss-Legendre of order Q_SELF in theta on each and in rho on
    [0, rho_hat(theta)].  D, S and K are weakly singular there (the curvature
    makes (x - y).n = O(rho^2)) and integrate directly.  H is hypersingular:
    with y - x = rho A + rho^2 B + O(rho^3) (A = y_xi cos + y_eta sin,
    B = (y_xixi cos^2 + 2 y_xieta cos sin + y_etaeta sin^2)/2 at the centre),
    beta = |A| and |J| = J0 + rho J1(theta) + O(rho^2), the integrand
    F = H |J| rho has the Laurent expansion F_-2 / rho^2 + F_-1 / rho + O(1),
        F_-2 = J0 / (4 pi beta^3),
        F_-1 = (J1 - 3 J0 (A.B)/beta^2) / (4 pi beta^3)
    (the (x-y).n_x (x-y).n_y / r^5 term is O(1); n_x.n_y = 1 + O(rho^2)).
    The Hadamard finite part with a spherical exclusion |y - x| < eps (its
    parameter radius is eps/beta - eps^2 (A.B)/beta^4 + O(eps^3)) is
        int_theta int_0^rho_hat (F - F_-2/rho^2 - F_-1/rho) drho dtheta
        + int_theta [F_-1 ln(rho_hat beta) + F_-2 ((A.B)/beta^2 - 1/rho_hat)] dtheta,
    the divergent eps^-1 part dropped and the ln(eps) part vanishing because
    F_-1(theta + pi) = -F_-1(theta).  For the centre of the symmetric
    parameter square the (A.B) and ln terms integrate to zero as well (both
    odd under theta -> theta + pi); they are kept for other collocation
    points.  On a flat element A.B = 0 and F_-1 = 0, and this is the closed
    form of bem.py.
"""
import numpy as np

from . import bem, fmm
from . import special as sp

Q_FAR4 = 4
Q_NEAR8 = 8
Q_SELF = 16


# ------------------------------------------------------------- geometry --

def _lag(t):
    """1-D quadratic Lagrange on -1, 0, 1: values, first and second derivatives."""
    t = np.asarray(t, dtype=np.float64)
    L = np.stack([0.5 * t * (t - 1.0), 1.0 - t * t, 0.5 * t * (t + 1.0)])
    dL = np.stack([t - 0.5, -2.0 * t, t + 0.5])
    d2L = np.stack([np.ones_like(t), -2.0 * np.ones_like(t), np.ones_like(t)])
    return L, dL, d2L


def shape(xi, eta):
    """N (9, ...), N_xi, N_eta, N_xixi, N_xieta, N_etaeta at the points."""
    L, dL, d2L = _lag(xi)
    M, dM, d2M = _lag(eta)
    out = []
    for A, Bm in ((L, M), (dL, M), (L, dM), (d2L, M), (dL, dM), (L, d2M)):
        out.append(np.stack([A[i] * Bm[j] for j in range(3) for i in range(3)]))
    return out


def geometry(Y, xi, eta):
    """y, y_xi, y_eta, y_xixi, y_xieta, y_etaeta (..., 3) of the element nodes Y (9 x 3)."""
    return [np.einsum("a...,ad->...d", Na, Y) for Na in shape(xi, eta)]


class Q9Mesh:
    def __init__(self, nodes, elems):
        self.nodes = np.asarray(nodes, dtype=np.float64)
        self.elems = np.asarray(elems, dtype=np.int64)
        self.Y = self.nodes[self.elems]                       # n x 9 x 3
        y, yx, ye = (a[:, 0] for a in _batch_geometry(self.Y, np.zeros(1), np.zeros(1)))
        J = np.cross(yx, ye)
        self.centroid = y                                     # collocation points
        self.normal = J / np.linalg.norm(J, axis=-1, keepdims=True)
        c = self.Y[:, [0, 2, 8, 6]]                           # corners in cyclic order
        self.hmax = np.max(np.linalg.norm(c - np.roll(c, 1, axis=1), axis=2), axis=1)
        self.n = len(self.elems)


def _gauss(q, a=-1.0, b=1.0):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def tensor_rule(q, box=(-1.0, 1.0, -1.0, 1.0)):
    xa, wa = _gauss(q, box[0], box[1])
    xb, wb = _gauss(q, box[2], box[3])
    XI, ETA = np.meshgrid(xa, xb, indexing="ij")
    return XI.ravel(), ETA.ravel(), np.outer(wa, wb).ravel()


def element_rule(Y, cls):
    """Points (P x 3), normals (P x 3), weights (P) of the regular class rule."""
    if cls == "far":
        rules = [tensor_rule(Q_FAR4)]
    elif cls == "near":
        rules = [tensor_rule(Q_NEAR8)]
    else:
        rules = [tensor_rule(Q_NEAR8, b) for b in ((-1, 0, -1, 0), (0, 1, -1, 0), (-1, 0, 0, 1), (0, 1, 0, 1))]
    xi = np.concatenate([r[0] for r in rules])
    eta = np.concatenate([r[1] for r in rules])
    w = np.concatenate([r[2] for r in rules])
    y, yx, ye = geometry(Y, xi, eta)[:3]
    J = np.cross(yx, ye)
    dJ = np.linalg.norm(J, axis=-1)
    return y, J / dJ[:, None], w * dJ


def pair_integrals(x, nx, Y, k, cls):
    """D, H, S, K of element nodes Y seen from (x, nx)."""
    y, ny, w = element_rule(Y, cls)
    D = np.sum(w * bem.kernel_dlp(x, nx, y, ny, k))
    H = np.sum(w * bem.kernel_hyp(x, nx, y, ny, k))
    S = np.sum(w * bem.kernel_slp(x, y, k))
    K = np.sum(w * bem.kernel_adlp(x, nx, y, k))
    return D, H, S, K


def _batch_geometry(Yb, xi, eta):
    """y, y_xi, y_eta (P x Q x 3) for P elements at Q parameter points."""
    N, Nx, Ne = shape(xi, eta)[:3]
    return [np.einsum("aq,pad->pqd", Na, Yb) for Na in (N, Nx, Ne)]


def _batch_rule(Yb, cls):
    if cls == "far":
        rules = [tensor_rule(Q_FAR4)]
    elif cls == "near":
        rules = [tensor_rule(Q_NEAR8)]
    else:
        rules = [tensor_rule(Q_NEAR8, b) for b in ((-1, 0, -1, 0), (0, 1, -1, 0), (-1, 0, 0, 1), (0, 1, 0, 1))]
    xi = np.concatenate([r[0] for r in rules])
    eta = np.concatenate([r[1] for r in rules])
    w = np.concatenate([r[2] for r in rules])
    y, yx, ye = _batch_geometry(Yb, xi, eta)
    J = np.cross(yx, ye)
    dJ = np.linalg.norm(J, axis=-1)
    return y, J / dJ[..., None], w[None, :] * dJ


# ------------------------------------------------------------ self terms --

def _polar_rule(q=Q_SELF):
    """Parameter-plane polar rule about (0, 0) on [-1, 1]^2: theta nodes and
    weights on the four sides' angular ranges, rho_hat(theta) to the side,
    and the rho nodes/weights on [0, 1] (to be scaled by rho_hat)."""
    ths, wts, rhat = [], [], []
    for c, (t0, t1) in enumerate(((-np.pi / 4, np.pi / 4), (np.pi / 4, 3 * np.pi / 4),
                                  (3 * np.pi / 4, 5 * np.pi / 4), (5 * np.pi / 4, 7 * np.pi / 4))):
        t, w = _gauss(q, t0, t1)
        ths.append(t)
        wts.append(w)
        rhat.append([1 / np.cos(t), 1 / np.sin(t), -1 / np.cos(t), -1 / np.sin(t)][c])
    u, wu = _gauss(q, 0.0, 1.0)
    return np.concatenate(ths), np.concatenate(wts), np.concatenate(rhat), u, wu


def self_integrals(Y, k, q=Q_SELF):
    """D, H (finite part), S, K of element Y (9 x 3) at its own centre."""
    th, wth, rhat, u, wu = _polar_rule(q)
    c, s = np.cos(th), np.sin(th)
    g = geometry(Y, 0.0, 0.0)
    y0, yx, ye, yxx, yxe, yee = g
    Jv = np.cross(yx, ye)
    J0 = np.linalg.norm(Jv)
    nx = Jv / J0
    # points (theta, rho)
    rho = rhat[:, None] * u[None, :]                      # T x U
    xi, eta = rho * c[:, None], rho * s[:, None]
    y, yxi, yeta = geometry(Y, xi, eta)[:3]
    J = np.cross(yxi, yeta)
    dJ = np.linalg.norm(J, axis=-1)
    ny = J / dJ[..., None]
    x = np.broadcast_to(y0, y.shape)
    nxb = np.broadcast_to(nx, y.shape)
    wgt = (wth[:, None] * wu[None, :] * rhat[:, None]) * rho * dJ   # polar Jacobian rho, area |J|
    D = np.sum(wgt * bem.kernel_dlp(x, nxb, y, ny, k))
    S = np.sum(wgt * bem.kernel_slp(x, y, k))
    K = np.sum(wgt * bem.kernel_adlp(x, nxb, y, k))
    # hypersingular finite part (Laurent coefficients of F = H |J| rho)
    A = yx[None, :] * c[:, None] + ye[None, :] * s[:, None]
    Bv = 0.5 * (yxx[None, :] * (c * c)[:, None] + 2 * yxe[None, :] * (c * s)[:, None] + yee[None, :] * (s * s)[:, None])
    beta = np.linalg.norm(A, axis=1)
    AB = np.einsum("ti,ti->t", A, Bv)
    Jx = np.cross(yxx, ye) + np.cross(yx, yxe)
    Je = np.cross(yxe, ye) + np.cross(yx, yee)
    J1 = (Jv[None, :] * (Jx[None, :] * c[:, None] + Je[None, :] * s[:, None])).sum(axis=1) / J0
    Fm2 = J0 / (4 * np.pi * beta ** 3)
    Fm1 = (J1 - 3 * J0 * AB / beta ** 2) / (4 * np.pi * beta ** 3)
    F = bem.kernel_hyp(x, nxb, y, ny, k) * dJ * rho
    inner = np.sum(wu[None, :] * rhat[:, None] * (F - Fm2[:, None] / rho ** 2 - Fm1[:, None] / rho), axis=1)
    H = np.sum(wth * (inner + Fm1 * np.log(rhat * beta) + Fm2 * (AB / beta ** 2 - 1 / rhat)))
    return D, H, S, K


# -------------------------------------------------------------- operator --

def dhsk_block(tgt: Q9Mesh, src_Y, k, self_pairs=None, chunk=4000):
    """D, H, S, K (n_t x n_s) of collocation points of tgt against source
    elements with nodes src_Y (n_s x 9 x 3, placed); self_pairs: boolean mask
    of pairs with x_i the centre of E_j."""
    nt_, ns = tgt.n, len(src_Y)
    ycen = _batch_geometry(src_Y, np.zeros(1), np.zeros(1))[0][:, 0]
    c = src_Y[:, [0, 2, 8, 6]]
    hmax = np.max(np.linalg.norm(c - np.roll(c, 1, axis=1), axis=2), axis=1)
    cls = bem.classify(tgt.centroid[:, None, :], ycen[None], hmax[None])
    if self_pairs is not None:
        cls[self_pairs] = 3
    out = [np.zeros((nt_, ns), dtype=complex) for _ in range(4)]
    names = {0: "far", 1: "near", 2: "verynear"}
    for cc in (0, 1, 2):
        ii, jj = np.nonzero(cls == cc)
        for s0 in range(0, len(ii), chunk):
            i, j = ii[s0:s0 + chunk], jj[s0:s0 + chunk]
            y, ny, w = _batch_rule(src_Y[j], names[cc])
            x = tgt.centroid[i][:, None, :]
            nx = tgt.normal[i][:, None, :]
            vals = (np.sum(w * bem.kernel_dlp(x, nx, y, ny, k), axis=1),
                    np.sum(w * bem.kernel_hyp(x, nx, y, ny, k), axis=1),
                    np.sum(w * bem.kernel_slp(x, y, k), axis=1),
                    np.sum(w * bem.kernel_adlp(x, nx, y, k), axis=1))
            for o, v in zip(out, vals):
                o[i, j] = v
    for i, j in zip(*np.nonzero(cls == 3)):
        for o, v in zip(out, self_integrals(src_Y[j], k)):
            o[i, j] = v
    return out


def dense_matrix(nodes, elems, k, beta=0.0):
    """The collocation matrix of Eq. (bm) on the Q9 mesh (one cell):
    A = (1/2 + beta/2) I - (D + b H) - i k beta (S + b K)."""
    m = Q9Mesh(nodes, elems)
    D, H, S, K = dhsk_block(m, m.Y, k, self_pairs=np.eye(m.n, dtype=bool))
    return (0.5 + 0.5 * beta) * np.eye(m.n) + bem._entries(D, H, S, K, k, beta)


def plane_wave_rhs(mesh: Q9Mesh, k, direction, amp=1.0):
    d = np.asarray(direction, dtype=np.float64)
    pinc = amp * np.exp(1j * k * (mesh.centroid @ d))
    return pinc + bem.coupling(k) * 1j * k * (mesh.normal @ d) * pinc


def toeplitz_block(cell: Q9Mesh, lattice, delta, k, beta=0.0):
    """T_delta of a periodic array of Q9 cells (Eq. (blockToeplizMatrix)):
    collocation points of the cell at the origin against the elements of the
    cell displaced by -delta . lattice."""
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    selfp = np.eye(cell.n, dtype=bool) if not np.any(delta) else None
    D, H, S, K = dhsk_block(cell, cell.Y + shift[None, None, :], k, self_pairs=selfp)
    T = bem._entries(D, H, S, K, k, beta)
    if selfp is not None:
        T += (0.5 + 0.5 * beta) * np.eye(cell.n)
    return T


# ------------------------------------------------------------ FMM tables --

def p2m_table(mesh: Q9Mesh, k, nt, beta=0.0):
    """V_0 (B x n) of Eq. (p2m) on the curved elements: the far-class rule
    (4 x 4 Gauss-Legendre) with the normal of each point, about the cell
    origin.  With an admittance the single-layer source term adds
    i k beta int conj(I_q) dA, as on flat triangles (fmm.p2m_table).  The
    L2P table needs only the collocation points and their normals:
    fmm.l2p_table(mesh, k, nt)."""
    y, ny, w = _batch_rule(mesh.Y, "far")                # n x 16 x 3, n x 16 x 3, n x 16
    g = sp.grad_regular_table(nt, y, k)                   # B x n x 16 x 3
    dIdn = np.einsum("bnqi,nqi->bnq", g, ny)
    V = np.sum(np.conj(dIdn) * w[None], axis=2)
    if beta != 0:
        I = sp.wave_table(nt, y.reshape(-1, 3), k, "I").reshape(-1, *w.shape)
        V = V + 1j * k * beta * np.sum(np.conj(I) * w[None], axis=2)
    return V


def fmm_matvec_explicit(mesh: Q9Mesh, lattice, counts, k, nt, p, beta=0.0):
    """The FMPBEM product (Eq. (2dPeriodicFMM)) on a Q9 cell, every cell
    pair explicitly: near blocks (|delta|_inf <= 1) from toeplitz_block,
    far pairs through U_0 K(delta) V_0."""
    near = {d: toeplitz_block(mesh, lattice, d, k, beta) for d in bem.near_offsets(counts)}
    return fmm.fmm_matvec_explicit(mesh, lattice, counts, k, nt, p, near_blocks=near,
                                   V0=p2m_table(mesh, k, nt, beta), U0=fmm.l2p_table(mesh, k, nt), beta=beta)


# ---------------------------------------------------------- FMPBEM2 near --
# The multilevel near field of fmm2.py on a Q9 cell: the octree of the
# element centres, the boxes' radii over the nine nodes of their elements,
# the leaf P2M table over the far-class rule with each point's normal, and
# the exact entries of P2P pairs from toeplitz_block.

class _Fmm2Cell:
    """A Q9Mesh under the names fmm2.py reads (centroid, normal, v, n)."""

    def __init__(self, mesh: Q9Mesh):
        self.mesh = mesh
        self.centroid, self.normal, self.v, self.n = mesh.centroid, mesh.normal, mesh.Y, mesh.n


def p2m_leaf(cell, elems, centre, k, nt, beta=0.0):
    """V (B x len(elems)) about a leaf centre (p2m_table's rule)."""
    y, ny, w = _batch_rule(cell.mesh.Y[elems], "far")
    rel = y - np.asarray(centre)[None, None, :]
    g = sp.grad_regular_table(nt, rel, k)
    V = np.sum(np.conj(np.einsum("bnqi,nqi->bnq", g, ny)) * w[None], axis=2)
    if beta != 0:
        I = sp.wave_table(nt, rel.reshape(-1, 3), k, "I").reshape(-1, *w.shape)
        V = V + 1j * k * beta * np.sum(np.conj(I) * w[None], axis=2)
    return V


def fmm2_near_block(mesh: Q9Mesh, lattice, delta, k, nt_near, levels, beta=0.0):
    """The multilevel approximation of S_delta (n x n) on a Q9 cell."""
    from . import fmm2
    cell = _Fmm2Cell(mesh)
    tree = fmm2.Octree(cell, levels)
    S = toeplitz_block(mesh, lattice, delta, k, beta)
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    return fmm2.near_block_apply(cell, tree, shift, k, nt_near, np.eye(mesh.n), S, beta, p2m=p2m_leaf).T


def fmm2_matvec_explicit(mesh: Q9Mesh, lattice, counts, k, nt, nt_near, levels, p, beta=0.0):
    """The FMPBEM2 product on a Q9 cell: fmm_matvec_explicit with every near
    block replaced by its multilevel approximation."""
    near = {d: fmm2_near_block(mesh, lattice, d, k, nt_near, levels, beta) for d in bem.near_offsets(counts)}
    return fmm.fmm_matvec_explicit(mesh, lattice, counts, k, nt, p, near_blocks=near,
                                   V0=p2m_table(mesh, k, nt, beta), U0=fmm.l2p_table(mesh, k, nt), beta=beta)

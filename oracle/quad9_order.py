"""Burton-Miller collocation on nine-node quadratic quadrilaterals with
discontinuous pressure of order 0, 1 or 2 (the paper's discontinuous
Lagrange pressure of variable order, Sec. 2.1 and Eq. (matrixBEM)).  Oracle
code: test infrastructure only.

Pressure on element f: p(y) = sum_b N_b(xi, eta) p_{f,b}, with nodes inside
the element (discontinuous: no node on an edge), collocated at the nodes
x_{f,a} = y_f(xi_a, eta_a) with the normal there:
  * order 0: one node at (0, 0), N = 1 (quad9.py's element);
  * order 1: 2 x 2 nodes at (+-s1, +-s1), s1 = 1/sqrt(3), bilinear Lagrange;
  * order 2: the eight-node serendipity element on [-s2, s2]^2,
    s2 = sqrt(3/5), nodes at the corners and side midpoints of that square.
The dof counts of the paper's h-study (8 pressure dofs per quadratic
element) fix the eight-node form of order 2; the node positions are not
printed and are taken at the Gauss-Legendre points of the matching order.

Entries (mesh normals into the fluid, b = i/k):
  A[(e,a),(f,b)] = 1/2 (1 + beta) [(e,a) = (f,b)]
                   - int_{E_f} N_b [dG/dn_y + b d2G/dn_x dn_y] dA
                   - i k beta int_{E_f} N_b [G + b dG/dn_x] dA,
x = x_{e,a}.  The 1/2 free term needs p smooth at x, which the
discontinuous element gives.

Rules.  Regular pairs by d = |x - y_f(0, 0)| against the longest corner
chord h_f: far d >= 4 h: 4 x 4 Gauss-Legendre; near 1.5 h <= d < 4 h: 8 x 8;
very near: 8 x 8 on each of 2 x 2 (order 0, quad9.py's rule), 4 x 4 (order
1) or 8 x 8 (order 2) parameter sub-squares: the collocation points of the
higher orders lie closer to the element edges (s2 puts them 0.11 h from the
neighbour), and these subdivisions keep the closed-surface identities at
about 1e-8 for every order.
Self pairs (x on E_f): polar coordinates about (xi_a, eta_a), the square cut
into four triangles with apex there, Q_SELF-point Gauss-Legendre in theta on
each triangle's angle range and in rho on [0, rho_hat(theta)], Q_SELF = 16
for order 0 (quad9.py's rule) and 24 for orders 1 and 2, whose off-centre
apex leaves thin triangles towards the nearest side.  D, S, K
directly; H as the Hadamard finite part with a spherical exclusion.  With
F = H |J| rho = F_-2/rho^2 + F_-1/rho + O(1) (quad9.py, now at (xi_a, eta_a))
and N_b = N_b0 + rho N_b1(theta) + O(rho^2) (N_b0 = N_b(xi_a, eta_a),
N_b1 = grad N_b . (cos, sin)), the product G = F N_b has
  G_-2 = F_-2 N_b0,   G_-1 = F_-1 N_b0 + F_-2 N_b1,
and the finite part is
  int_theta int_0^rho_hat (G - G_-2/rho^2 - G_-1/rho) drho dtheta
  + int_theta [G_-1 ln(rho_hat beta) + G_-2 ((A.B)/beta^2 - 1/rho_hat)] dtheta;
G_-1 is odd under theta -> theta + pi, so the ln(eps) part vanishes.  Away
from the centre the (A.B) and ln terms do not cancel.
"""
import numpy as np

from . import bem, quad9

S1 = 1.0 / np.sqrt(3.0)
S2 = np.sqrt(3.0 / 5.0)
Q_SELF = (16, 24, 24)     # self-rule order by pressure order (16: quad9.py's rule)


class PressureBasis:
    """Discontinuous pressure shape functions of one order on [-1, 1]^2."""

    def __init__(self, order: int):
        if order not in (0, 1, 2):
            raise ValueError("pressure order must be 0, 1 or 2")
        self.order = order
        if order == 0:
            self.nodes = np.zeros((1, 2))
        elif order == 1:
            self.nodes = np.array([[-S1, -S1], [S1, -S1], [-S1, S1], [S1, S1]])
        else:
            u = np.array([[-1, -1], [0, -1], [1, -1], [1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0]], dtype=float)
            self.nodes = S2 * u
        self.nb = len(self.nodes)

    def eval(self, xi, eta):
        """N (nb, ...) and grad N (nb, 2, ...) with respect to (xi, eta)."""
        xi, eta = np.broadcast_arrays(np.asarray(xi, dtype=float), np.asarray(eta, dtype=float))
        if self.order == 0:
            N = np.ones((1,) + xi.shape)
            return N, np.zeros((1, 2) + xi.shape)
        if self.order == 1:
            l = [(S1 - xi) / (2 * S1), (S1 + xi) / (2 * S1)]
            m = [(S1 - eta) / (2 * S1), (S1 + eta) / (2 * S1)]
            dl = [-np.ones_like(xi) / (2 * S1), np.ones_like(xi) / (2 * S1)]
            dm = [-np.ones_like(eta) / (2 * S1), np.ones_like(eta) / (2 * S1)]
            N, G = [], []
            for j in range(2):
                for i in range(2):
                    N.append(l[i] * m[j])
                    G.append(np.stack([dl[i] * m[j], l[i] * dm[j]]))
            return np.stack(N), np.stack(G)
        u, v = xi / S2, eta / S2
        N, G = [], []
        for ua, va in self.nodes / S2:
            if ua != 0 and va != 0:
                N.append(0.25 * (1 + u * ua) * (1 + v * va) * (u * ua + v * va - 1))
                du = 0.25 * ua * (1 + v * va) * (2 * u * ua + v * va)
                dv = 0.25 * va * (1 + u * ua) * (u * ua + 2 * v * va)
            elif ua == 0:
                N.append(0.5 * (1 - u * u) * (1 + v * va))
                du = -u * (1 + v * va)
                dv = 0.5 * va * (1 - u * u)
            else:
                N.append(0.5 * (1 + u * ua) * (1 - v * v))
                du = 0.5 * ua * (1 - v * v)
                dv = -v * (1 + u * ua)
            G.append(np.stack([du / S2, dv / S2]))
        return np.stack(N), np.stack(G)


class OrderMesh:
    """A Q9 mesh with a pressure basis: collocation points and normals of
    every (element, node), dof index e * nb + a."""

    def __init__(self, nodes, elems, order):
        self.geo = quad9.Q9Mesh(nodes, elems)
        self.basis = PressureBasis(order)
        self.n = self.geo.n
        self.nb = self.basis.nb
        nd = self.basis.nodes
        y, yx, ye = quad9._batch_geometry(self.geo.Y, nd[:, 0], nd[:, 1])
        J = np.cross(yx, ye)
        self.points = y.reshape(-1, 3)
        self.normals = (J / np.linalg.norm(J, axis=-1, keepdims=True)).reshape(-1, 3)


def _rule(cls, order):
    if cls == 0:
        return quad9.tensor_rule(quad9.Q_FAR4)
    if cls == 1:
        return quad9.tensor_rule(quad9.Q_NEAR8)
    parts = (2, 4, 8)[order]
    edges = np.linspace(-1.0, 1.0, parts + 1)
    rules = [quad9.tensor_rule(quad9.Q_NEAR8, (edges[i], edges[i + 1], edges[j], edges[j + 1]))
             for j in range(parts) for i in range(parts)]
    return tuple(np.concatenate([r[q] for r in rules]) for q in range(3))


def _polar_rule(xa, ea, q):
    """theta nodes, weights, rho_hat(theta) of the four triangles about
    (xa, ea), and the rho nodes/weights on [0, 1]."""
    corners = [(1.0, -1.0), (1.0, 1.0), (-1.0, 1.0), (-1.0, -1.0)]
    ang = [np.arctan2(cy - ea, cx - xa) for cx, cy in corners]
    for i in range(1, 4):
        while ang[i] <= ang[i - 1]:
            ang[i] += 2 * np.pi
    ang.append(ang[0] + 2 * np.pi)
    ths, wts, rh = [], [], []
    for side in range(4):
        t, w = quad9._gauss(q, ang[side], ang[side + 1])
        c, s = np.cos(t), np.sin(t)
        rhat = [(1.0 - xa) / c, (1.0 - ea) / s, (-1.0 - xa) / c, (-1.0 - ea) / s][side]
        ths.append(t)
        wts.append(w)
        rh.append(rhat)
    u, wu = quad9._gauss(q, 0.0, 1.0)
    return np.concatenate(ths), np.concatenate(wts), np.concatenate(rh), u, wu


def self_integrals(Y, basis: PressureBasis, a, k, q=None):
    """D, H (finite part), S, K (each nb values: one per source shape N_b)
    of element Y at its own collocation node a; q: self-rule order (default
    Q_SELF[order])."""
    q = Q_SELF[basis.order] if q is None else q
    xa, ea = basis.nodes[a]
    th, wth, rhat, u, wu = _polar_rule(xa, ea, q)
    c, s = np.cos(th), np.sin(th)
    y0, yx, ye, yxx, yxe, yee = quad9.geometry(Y, xa, ea)
    Jv = np.cross(yx, ye)
    J0 = np.linalg.norm(Jv)
    nx = Jv / J0
    rho = rhat[:, None] * u[None, :]
    xi, eta = xa + rho * c[:, None], ea + rho * s[:, None]
    y, yxi, yeta = quad9.geometry(Y, xi, eta)[:3]
    J = np.cross(yxi, yeta)
    dJ = np.linalg.norm(J, axis=-1)
    ny = J / dJ[..., None]
    x = np.broadcast_to(y0, y.shape)
    nxb = np.broadcast_to(nx, y.shape)
    N, _ = basis.eval(xi, eta)                                     # nb x T x U
    N0, G0 = basis.eval(np.array(xa), np.array(ea))                # nb, nb x 2
    wgt = (wth[:, None] * wu[None, :] * rhat[:, None]) * rho * dJ
    kd = bem.kernel_dlp(x, nxb, y, ny, k)
    ks = bem.kernel_slp(x, y, k)
    kk = bem.kernel_adlp(x, nxb, y, k)
    D = np.einsum("btu,tu->b", N, wgt * kd)
    S = np.einsum("btu,tu->b", N, wgt * ks)
    K = np.einsum("btu,tu->b", N, wgt * kk)
    A = yx[None, :] * c[:, None] + ye[None, :] * s[:, None]
    Bv = 0.5 * (yxx[None, :] * (c * c)[:, None] + 2 * yxe[None, :] * (c * s)[:, None] + yee[None, :] * (s * s)[:, None])
    beta = np.linalg.norm(A, axis=1)
    AB = np.einsum("ti,ti->t", A, Bv)
    Jx = np.cross(yxx, ye) + np.cross(yx, yxe)
    Je = np.cross(yxe, ye) + np.cross(yx, yee)
    J1 = (Jv[None, :] * (Jx[None, :] * c[:, None] + Je[None, :] * s[:, None])).sum(axis=1) / J0
    Fm2 = J0 / (4 * np.pi * beta ** 3)
    Fm1 = (J1 - 3 * J0 * AB / beta ** 2) / (4 * np.pi * beta ** 3)
    Nb0 = N0.reshape(-1)                                           # nb
    Nb1 = G0[:, 0].reshape(-1, 1) * c[None, :] + G0[:, 1].reshape(-1, 1) * s[None, :]   # nb x T
    Gm2 = Fm2[None, :] * Nb0[:, None]
    Gm1 = Fm1[None, :] * Nb0[:, None] + Fm2[None, :] * Nb1
    F = bem.kernel_hyp(x, nxb, y, ny, k) * dJ * rho                # T x U
    G = N * F[None]
    inner = np.sum(wu[None, None, :] * rhat[None, :, None]
                   * (G - Gm2[:, :, None] / rho[None] ** 2 - Gm1[:, :, None] / rho[None]), axis=2)
    H = np.sum(wth[None, :] * (inner + Gm1 * np.log(rhat * beta)[None, :]
                               + Gm2 * (AB / beta ** 2 - 1 / rhat)[None, :]), axis=1)
    return D, H, S, K


def dhsk_block(tgt: OrderMesh, src_Y, k, self_same=False, chunk=2000):
    """D, H, S, K ((n nb) x (n_s nb)) of tgt's collocation points against
    the elements src_Y (placed); self_same: src_Y is tgt's own cell at its
    own place, so that a point's own element takes the self rule."""
    nb = tgt.nb
    basis = tgt.basis
    ns = len(src_Y)
    ycen = src_Y[:, 4]
    c = src_Y[:, [0, 2, 8, 6]]
    hmax = np.max(np.linalg.norm(c - np.roll(c, 1, axis=1), axis=2), axis=1)
    X, NX = tgt.points, tgt.normals
    cls = bem.classify(X[:, None, :], ycen[None], hmax[None])     # (n nb) x ns
    if self_same:
        for e in range(tgt.n):
            cls[e * nb:(e + 1) * nb, e] = 3
    out = [np.zeros((len(X), ns * nb), dtype=complex) for _ in range(4)]
    for cc in (0, 1, 2):
        xi, eta, w = _rule(cc, basis.order)
        N, _ = basis.eval(xi, eta)                                # nb x P
        Nq, Nx, Ne = quad9.shape(xi, eta)[:3]
        ii, jj = np.nonzero(cls == cc)
        for s0 in range(0, len(ii), chunk):
            i, j = ii[s0:s0 + chunk], jj[s0:s0 + chunk]
            Yb = src_Y[j]
            y = np.einsum("ap,qad->qpd", Nq, Yb)
            yx = np.einsum("ap,qad->qpd", Nx, Yb)
            ye = np.einsum("ap,qad->qpd", Ne, Yb)
            J = np.cross(yx, ye)
            dJ = np.linalg.norm(J, axis=-1)
            ny = J / dJ[..., None]
            wq = w[None, :] * dJ
            x = X[i][:, None, :]
            nx = NX[i][:, None, :]
            vals = (wq * bem.kernel_dlp(x, nx, y, ny, k), wq * bem.kernel_hyp(x, nx, y, ny, k),
                    wq * bem.kernel_slp(x, y, k), wq * bem.kernel_adlp(x, nx, y, k))
            for o, v in zip(out, vals):
                ent = v @ N.T                                      # pairs x nb
                for b in range(nb):
                    o[i, j * nb + b] = ent[:, b]
    for r, f in zip(*np.nonzero(cls == 3)):
        a = r - f * nb
        for o, v in zip(out, self_integrals(src_Y[f], basis, a, k)):
            o[r, f * nb:(f + 1) * nb] = v
    return out


def dense_matrix(nodes, elems, order, k, beta=0.0):
    """Collocation matrix of Eq. (bm) on one mesh (dof e nb + a)."""
    m = OrderMesh(nodes, elems, order)
    D, H, S, K = dhsk_block(m, m.geo.Y, k, self_same=True)
    return (0.5 + 0.5 * beta) * np.eye(m.n * m.nb) + bem._entries(D, H, S, K, k, beta)


def plane_wave_rhs(mesh: OrderMesh, k, direction, amp=1.0):
    d = np.asarray(direction, dtype=np.float64)
    pinc = amp * np.exp(1j * k * (mesh.points @ d))
    return pinc + bem.coupling(k) * 1j * k * (mesh.normals @ d) * pinc


def toeplitz_block(cell: OrderMesh, lattice, delta, k, beta=0.0):
    """T_delta (Eq. (blockToeplizMatrix)): the cell's collocation points
    against its elements displaced by -delta . lattice."""
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    same = not np.any(delta)
    D, H, S, K = dhsk_block(cell, cell.geo.Y + shift[None, None, :], k, self_same=same)
    T = bem._entries(D, H, S, K, k, beta)
    if same:
        T += (0.5 + 0.5 * beta) * np.eye(cell.n * cell.nb)
    return T


# ------------------------------------------------------------ FMM tables --

class _Colloc:
    """The collocation points of an OrderMesh under the names fmm.l2p_table reads."""

    def __init__(self, mesh: OrderMesh):
        self.centroid, self.normal = mesh.points, mesh.normals


def p2m_table(mesh: OrderMesh, k, nt, beta=0.0, dsign=1.0):
    """V_0 (B x n nb) of Eq. (p2m) with the pressure shapes: column f nb + b
    integrates N_b conj(dI_q/dn_y) (+ i k beta N_b conj(I_q)) over element f
    with the far-class rule (4 x 4 Gauss-Legendre), each point's normal;
    dsign = -1 for a mirrored cell whose nodes kept their order (its computed
    normal is -R n: only the double-layer term changes sign)."""
    xi, eta, w0 = quad9.tensor_rule(quad9.Q_FAR4)
    y, ny, w = quad9._batch_rule(mesh.geo.Y, "far")        # n x 16 x 3, n x 16 x 3, n x 16
    N, _ = mesh.basis.eval(xi, eta)                          # nb x 16
    from . import special as sp
    g = sp.grad_regular_table(nt, y, k)                      # B x n x 16 x 3
    src = dsign * np.conj(np.einsum("bnqi,nqi->bnq", g, ny))
    if beta != 0:
        I = sp.wave_table(nt, y.reshape(-1, 3), k, "I").reshape(-1, *w.shape)
        src = src + 1j * k * beta * np.conj(I)
    V = np.einsum("bnq,nq,cq->bnc", src, w, N)               # B x n x nb
    return V.reshape(V.shape[0], -1)


def fmm_matvec_explicit(mesh: OrderMesh, lattice, counts, k, nt, p, beta=0.0):
    """The FMPBEM product (Eq. (2dPeriodicFMM)) on a cell with pressure of
    any order, every cell pair explicitly: near blocks (|delta|_inf <= 1)
    from toeplitz_block, far pairs through U_0 K(delta) V_0."""
    from . import fmm
    near = {d: toeplitz_block(mesh, lattice, d, k, beta) for d in bem.near_offsets(counts)}

    class _Cell:
        n = mesh.n * mesh.nb

    return fmm.fmm_matvec_explicit(_Cell(), lattice, counts, k, nt, p, near_blocks=near,
                                   V0=p2m_table(mesh, k, nt, beta), U0=fmm.l2p_table(_Colloc(mesh), k, nt),
                                   beta=beta)


# ---------------------------------------------------------- field points --

def field_points(nodes, elems, order, lattice, counts, k, p, points, direction, amp=1.0, beta=0.0):
    """Total pressure in the fluid (Eq. (cbie) with c = 1) from the surface
    pressure p (dof (c n + e) nb + a over the cells of the array):
      p(x) = p_inc(x) + sum_{f,b} int_{E_f} N_b [dG/dn_y + i k beta G] dA p_{f,b},
    the single layer of dp/dn_m = -i k beta p joining the double layer with an
    admittance; the same class rules as the collocation points, by the
    distance of x to each element's centre."""
    from types import SimpleNamespace
    L = np.asarray(lattice, dtype=np.float64)
    nodes = np.asarray(nodes, dtype=np.float64)
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, dtype=np.float64) @ L for c in cells])
    allE = np.concatenate([np.asarray(elems) + i * len(nodes) for i in range(len(cells))])
    Y = allN[allE]
    basis = PressureBasis(order)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    tgt = SimpleNamespace(points=pts, normals=np.tile([0.0, 0.0, 1.0], (len(pts), 1)), basis=basis,
                          nb=basis.nb, n=0)
    D, _, S, _ = dhsk_block(tgt, Y, k)
    out = amp * np.exp(1j * k * (pts @ np.asarray(direction, dtype=np.float64)))
    return out + (D + 1j * k * beta * S) @ np.asarray(p)


# ------------------------------------------------------------- half-space --
# Eq. (green3dHalf): G_h(x, y) = G(x, y) + R_p G(x, y^).  The image
# integrals over element E_f are integrals over y^ = M y(xi, eta) with the
# normal R n(xi, eta) and the same area element and shapes N_b(xi, eta).  The
# mirrored nodes are kept in their order, so that the shapes keep their
# parameters; the Jacobian of the mirrored map is then -R J (a reflection
# reverses orientation), so the computed normal is -R n and the terms linear
# in n_y (D and H) change sign, while S and K (dG/dn_x) do not.  Shifts,
# lattice roles and the block Hankel part are those of halfspace.py.

def _image_entries(tgt, src_Y_mirrored, k, beta, Rp):
    D, H, S, K = dhsk_block(tgt, src_Y_mirrored, k)
    return Rp * bem._entries(-D, -H, S, K, k, beta)


def image_block(cell: OrderMesh, lattice, counts, plane, dt, k, beta=0.0):
    """T^(delta~): R_p times the entries of the cell's collocation points
    against the reflected unit cell (R Y) shifted by shift(delta~)."""
    from . import halfspace
    src = plane.reflect(cell.geo.Y) + halfspace.image_shift(lattice, counts, plane, dt)[None, None, :]
    return _image_entries(cell, src, k, beta, plane.Rp)


def dense_matrix_halfspace(nodes, elems, order, lattice, counts, k, plane, beta=0.0):
    """The dense collocation matrix of the whole array with G_h, pair by pair
    over the array and its mirror image, without any structure."""
    L = np.asarray(lattice, dtype=np.float64)
    cells = bem.lattice_cells(counts)
    nodes = np.asarray(nodes, dtype=np.float64)
    allN = np.concatenate([nodes + np.asarray(c, dtype=np.float64) @ L for c in cells])
    allE = np.concatenate([np.asarray(elems) + i * len(nodes) for i in range(len(cells))])
    m = OrderMesh(allN, allE, order)
    A = dense_matrix(allN, allE, order, k, beta)
    return A + _image_entries(m, plane.mirror(m.geo.Y), k, beta, plane.Rp)


def structured_matvec_halfspace(cell: OrderMesh, lattice, counts, k, plane, p, beta=0.0):
    """(T + T^) p as two block Toeplitz products (Sec. 2.4): T p, and
    (T^ P)(P p) with the cells reversed along the axis perpendicular to the
    plane (none: P = identity)."""
    from . import halfspace
    p = np.atleast_2d(p)
    h = halfspace.hankel_axis(lattice, counts, plane)
    blocks = {d: toeplitz_block(cell, lattice, d, k, beta) for d in bem.all_offsets(counts)}
    image = {d: image_block(cell, lattice, counts, plane, d, k, beta) for d in bem.all_offsets(counts)}
    return (bem.toeplitz_matvec(blocks, counts, p)
            + bem.toeplitz_matvec(image, counts, halfspace.reverse_cells(p, counts, h)))


def incident_with_image(mesh: OrderMesh, k, direction, plane, amp=1.0):
    """b = p_inc + b dp_inc/dn at the collocation points for the plane wave
    amp e^{i k d.x} with its image R_p p_inc(M x)."""
    d = np.asarray(direction, dtype=np.float64)
    X, Nn = mesh.points, mesh.normals
    p1 = amp * np.exp(1j * k * (X @ d))
    dp1 = 1j * k * (Nn @ d) * p1
    Xm, Nm = plane.mirror(X), plane.reflect(Nn)
    p2 = amp * np.exp(1j * k * (Xm @ d))
    dp2 = 1j * k * (Nm @ d) * p2
    return (p1 + plane.Rp * p2) + bem.coupling(k) * (dp1 + plane.Rp * dp2)


def field_points_halfspace(nodes, elems, order, lattice, counts, k, p, points, direction, plane, amp=1.0,
                           beta=0.0):
    """field_points with G_h: the incident wave and its image
    R_p p_inc(M x), plus R_p times the surface's mirrored contribution (the
    mirrored nodes in their order: D changes sign, S does not)."""
    from types import SimpleNamespace
    L = np.asarray(lattice, dtype=np.float64)
    nodes = np.asarray(nodes, dtype=np.float64)
    cells = bem.lattice_cells(counts)
    allN = np.concatenate([nodes + np.asarray(c, dtype=np.float64) @ L for c in cells])
    allE = np.concatenate([np.asarray(elems) + i * len(nodes) for i in range(len(cells))])
    Y = allN[allE]
    basis = PressureBasis(order)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    tgt = SimpleNamespace(points=pts, normals=np.tile([0.0, 0.0, 1.0], (len(pts), 1)), basis=basis,
                          nb=basis.nb, n=0)
    d = np.asarray(direction, dtype=np.float64)
    out = amp * (np.exp(1j * k * (pts @ d)) + plane.Rp * np.exp(1j * k * (plane.mirror(pts) @ d)))
    D, _, S, _ = dhsk_block(tgt, Y, k)
    Dm, _, Sm, _ = dhsk_block(tgt, plane.mirror(Y), k)
    p = np.asarray(p)
    return out + (D + 1j * k * beta * S) @ p + plane.Rp * ((-Dm + 1j * k * beta * Sm) @ p)


def fmm_image_matvec_explicit(cell: OrderMesh, lattice, counts, k, nt, plane, p, beta=0.0):
    """The image part of Eq. (2dPeriodicFMM_halfspace), (S^ + U K^ V^) p, over
    every (target cell, mirrored source cell) pair (halfspace.py's near set
    and M2L translations): near pairs by image_block, far pairs through
    U_0 K^ V^ with V^ = R_p times the P2M table of the reflected cell."""
    from . import fmm, halfspace
    p = np.atleast_2d(p)
    h = halfspace.hankel_axis(lattice, counts, plane)
    q = halfspace.reverse_cells(p, counts, h)
    cells = bem.lattice_cells(counts)
    n = cell.n * cell.nb
    R = p.shape[0]
    Q = q.reshape(R, len(cells), n)
    near = set(halfspace.image_near_offsets(lattice, counts, plane))
    refl = OrderMesh(plane.reflect(cell.geo.nodes), cell.geo.elems, cell.basis.order)
    V0h = plane.Rp * p2m_table(refl, k, nt, beta, dsign=-1.0)
    U0 = fmm.l2p_table(_Colloc(cell), k, nt)
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
                    cache[key] = fmm.m2l_block(-halfspace.image_shift(lattice, counts, plane, dt), k, nt)
                Lc += Mom[:, cj] @ cache[key].T
        Y[:, ci] += Lc @ U0.T
    return Y.reshape(R, -1)


# ---------------------------------------------------------- FMPBEM2 near --
# fmm2.py's multilevel near field on a cell with pressure of any order: the
# octree of the element centres (box radii over the nine nodes), leaf P2M
# tables weighted by the shapes, leaf L2P tables at the elements' nodes, and
# dofs e nb + a of each leaf element.

class _Fmm2Cell:
    def __init__(self, mesh: OrderMesh):
        self.mesh = mesh
        self.centroid, self.v, self.n = mesh.geo.centroid, mesh.geo.Y, mesh.geo.n


def _leaf_p2m(cell, elems, centre, k, nt, beta=0.0):
    from . import special as sp
    mesh = cell.mesh
    xi, eta, _ = quad9.tensor_rule(quad9.Q_FAR4)
    y, ny, w = quad9._batch_rule(mesh.geo.Y[elems], "far")
    N, _ = mesh.basis.eval(xi, eta)
    rel = y - np.asarray(centre)[None, None, :]
    g = sp.grad_regular_table(nt, rel, k)
    src = np.conj(np.einsum("bnqi,nqi->bnq", g, ny))
    if beta != 0:
        src = src + 1j * k * beta * np.conj(sp.wave_table(nt, rel.reshape(-1, 3), k, "I").reshape(-1, *w.shape))
    return np.einsum("bnq,nq,cq->bnc", src, w, N).reshape(src.shape[0], -1)


def _leaf_l2p(cell, elems, centre, k, nt):
    from . import fmm2
    from types import SimpleNamespace
    mesh, nb = cell.mesh, cell.mesh.nb
    d = np.array([e * nb + a for e in elems for a in range(nb)])
    pts = SimpleNamespace(centroid=mesh.points[d], normal=mesh.normals[d])
    return fmm2.l2p_leaf(pts, np.arange(len(d)), centre, k, nt)


def fmm2_near_block(mesh: OrderMesh, lattice, delta, k, nt_near, levels, beta=0.0):
    """The multilevel approximation of S_delta ((n nb) x (n nb))."""
    from . import fmm2
    cell = _Fmm2Cell(mesh)
    tree = fmm2.Octree(cell, levels)
    S = toeplitz_block(mesh, lattice, delta, k, beta)
    shift = -np.asarray(delta, dtype=np.float64) @ np.asarray(lattice, dtype=np.float64)
    nb = mesh.nb
    dofs = lambda el: np.array([e * nb + a for e in el for a in range(nb)], dtype=np.int64)
    return fmm2.near_block_apply(cell, tree, shift, k, nt_near, np.eye(mesh.n * nb), S, beta,
                                 p2m=_leaf_p2m, l2p=_leaf_l2p, dofs=dofs).T

"""Unit-cell surface meshes of flat triangles, wound so that the right-hand
normal (v1 - v0) x (v2 - v0) points out of the body into the fluid.

Every mesh is centred on the origin, which is also the expansion centre of the
cell.  Shapes follow the synthetic stand-ins for the paper's scatterers
(spheres of the array study, cylinders of the sonic-crystal barrier of the
sound-barrier study, cubes for a 3-D lattice).
"""
import numpy as np


def _orient_outward(verts, tris):
    """Flip every triangle whose normal points towards the origin (all three
    shapes are star-shaped about the origin, so this gives outward normals)."""
    v = verts[tris]
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    cen = v.mean(axis=1)
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def icosphere(level: int, radius: float):
    """Icosahedron (12 vertices: cyclic permutations of (0, +-1, +-phi)),
    refined ``level`` times by splitting each triangle into four with edge
    midpoints pushed out to the sphere.  Level 2 has 320 triangles."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    base = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            base += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    verts = np.array(base, dtype=np.float64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    # faces: every triple of mutually nearest vertices (edge length 2 before scaling)
    d = np.linalg.norm(verts[:, None] - verts[None], axis=2)
    edge = d[d > 1e-9].min()
    adj = np.abs(d - edge) < 1e-9
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    tris = np.array(faces, dtype=np.int64)
    vlist = [tuple(v) for v in verts]
    for _ in range(level):
        cache = {}
        vlist_arr = vlist

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = (np.array(vlist_arr[a]) + np.array(vlist_arr[b])) / 2.0
                m /= np.linalg.norm(m)
                vlist_arr.append(tuple(m))
                cache[key] = len(vlist_arr) - 1
            return cache[key]

        new = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = np.array(new, dtype=np.int64)
    verts = np.array(vlist, dtype=np.float64) * radius
    tris = _orient_outward(verts, tris)
    return verts, tris.astype(np.int32)


def capped_cylinder(radius: float, height: float, n_around: int = 20, n_rows: int = 29):
    """Closed cylinder along z, centred on the origin: ``n_around`` segments
    by ``n_rows`` rows of side quads (two triangles each) plus a triangle fan
    of ``n_around`` triangles on each cap.  With the defaults: 1,160 side and
    40 cap triangles, 1,200 in total."""
    ang = 2.0 * np.pi * np.arange(n_around) / n_around
    zs = np.linspace(-height / 2.0, height / 2.0, n_rows + 1)
    verts = []
    for z in zs:
        for a in ang:
            verts.append((radius * np.cos(a), radius * np.sin(a), z))
    bottom = len(verts)
    verts.append((0.0, 0.0, -height / 2.0))
    top = len(verts)
    verts.append((0.0, 0.0, height / 2.0))
    tris = []
    for r in range(n_rows):
        for s in range(n_around):
            a = r * n_around + s
            b = r * n_around + (s + 1) % n_around
            c = (r + 1) * n_around + s
            d = (r + 1) * n_around + (s + 1) % n_around
            tris += [(a, b, d), (a, d, c)]
    for s in range(n_around):
        tris.append((bottom, (s + 1) % n_around, s))
        tris.append((top, n_rows * n_around + s, n_rows * n_around + (s + 1) % n_around))
    verts = np.array(verts, dtype=np.float64)
    tris = _orient_outward(verts, np.array(tris, dtype=np.int64))
    return verts, tris.astype(np.int32)


def open_cylinder(radius: float, height: float, n_around: int = 12, n_rows: int = 14):
    """Mantle of a cylinder along z, centred on the origin, without caps (a
    unit cell of a column of stacked cells): ``n_around`` segments by
    ``n_rows`` rows of quads split into two triangles, wound so that the
    normals point radially outward (336 triangles with the defaults)."""
    ang = 2.0 * np.pi * np.arange(n_around) / n_around
    zs = np.linspace(-height / 2.0, height / 2.0, n_rows + 1)
    verts = np.array([(radius * np.cos(a), radius * np.sin(a), z) for z in zs for a in ang], dtype=np.float64)
    tris = []
    for r in range(n_rows):
        for s in range(n_around):
            a = r * n_around + s
            b = r * n_around + (s + 1) % n_around
            c = (r + 1) * n_around + s
            d = (r + 1) * n_around + (s + 1) % n_around
            tris += [(a, b, d), (a, d, c)]
    tris = np.array(tris, dtype=np.int64)
    v = verts[tris]
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    cen = v.mean(axis=1)
    flip = np.einsum("ij,ij->i", nrm[:, :2], cen[:, :2]) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris.astype(np.int32)


def quad9_sphere(m: int, radius: float):
    """Sphere of 6 m^2 nine-node quadratic quadrilaterals: each face of the
    cube [-1, 1]^3 split into m x m squares, the (2m + 1)^2 nodes of a face
    projected radially onto the sphere (shared nodes merged).  Returns
    (nodes, elements): elements (6 m^2 x 9) list their nodes in a 3 x 3 grid,
    node (i, j) at 3 j + i with i along xi and j along eta, oriented so that
    d y/d xi x d y/d eta points out of the sphere."""
    index, nodes, elems = {}, [], []

    def node(p):
        q = np.asarray(p, dtype=np.float64)
        q = q / np.linalg.norm(q) * radius
        key = tuple(np.round(q / radius * 1e9).astype(np.int64))
        if key not in index:
            index[key] = len(nodes)
            nodes.append(q)
        return index[key]

    g = np.linspace(-1.0, 1.0, 2 * m + 1)
    for axis in range(3):
        for sign in (-1.0, 1.0):
            a1, a2 = [d for d in range(3) if d != axis]
            for ey in range(m):
                for ex in range(m):
                    ids = []
                    for j in range(3):
                        for i in range(3):
                            p = np.zeros(3)
                            p[axis] = sign
                            p[a1] = g[2 * ex + i]
                            p[a2] = g[2 * ey + j]
                            ids.append(node(p))
                    elems.append(ids)
    nodes = np.array(nodes)
    elems = np.array(elems, dtype=np.int64)
    # orientation from the corner diagonals (the centre normal of the map)
    y = nodes[elems]
    dxi = y[:, 5] - y[:, 3]
    deta = y[:, 7] - y[:, 1]
    flip = np.einsum("ij,ij->i", np.cross(dxi, deta), y[:, 4]) < 0
    order = np.array([2, 1, 0, 5, 4, 3, 8, 7, 6])    # xi -> -xi
    elems[flip] = elems[flip][:, order]
    return nodes, elems.astype(np.int32)


def cube(edge: float, n_per_edge: int = 6):
    """Axis-aligned cube centred on the origin, each face an
    ``n_per_edge`` x ``n_per_edge`` grid of squares split into two triangles
    (432 triangles for the default 6)."""
    h = edge / 2.0
    t = np.linspace(-h, h, n_per_edge + 1)
    verts, index, tris = [], {}, []

    def vid(p):
        key = tuple(np.round(np.array(p) / edge * 4 * n_per_edge).astype(int))
        if key not in index:
            index[key] = len(verts)
            verts.append(tuple(p))
        return index[key]

    for axis in range(3):
        for sign in (-1.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(n_per_edge):
                for j in range(n_per_edge):
                    quad = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0.0, 0.0, 0.0]
                        p[axis] = sign * h
                        p[u_ax] = t[i + di]
                        p[v_ax] = t[j + dj]
                        quad.append(vid(p))
                    tris += [(quad[0], quad[1], quad[2]), (quad[0], quad[2], quad[3])]
    verts = np.array(verts, dtype=np.float64)
    tris = _orient_outward(verts, np.array(tris, dtype=np.int64))
    return verts, tris.astype(np.int32)


def mesh_signed_volume(verts, tris) -> float:
    """Enclosed volume by the divergence theorem; positive when every triangle
    normal points outward."""
    v = verts[tris]
    return float(np.einsum("ij,ij->i", v[:, 0], np.cross(v[:, 1], v[:, 2])).sum() / 6.0)

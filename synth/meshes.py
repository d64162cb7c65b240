"""Procedural closed triangle meshes with outward counter-clockwise orientation.

Every generator returns ``(xyz, tri)``: ``xyz`` is a float64 array [nv, 3] and
``tri`` an int32 array [nt, 3] whose vertex order is counter-clockwise when
seen from outside the closed surface (so the right-hand normal points out).
"""

import numpy as np


def _orient_outward(xyz, tri, inside_point):
    """Flip triangles whose right-hand normal points towards ``inside_point``."""
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    c = (v0 + v1 + v2) / 3.0
    flip = np.einsum("ij,ij->i", nrm, c - inside_point) < 0
    out = tri.copy()
    out[flip, 1], out[flip, 2] = tri[flip, 2], tri[flip, 1]
    return out


def icosphere(level, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Icosahedron refined ``level`` times by midpoint splitting, projected on a sphere.

    Triangles: 20 * 4**level (level 3 -> 1280, level 5 -> 20480).
    """
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
         [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
         [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    verts = [tuple(x) for x in v]
    for _ in range(level):
        cache = {}
        nf = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                m /= np.linalg.norm(m)
                cache[key] = len(verts)
                verts.append(tuple(m))
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    xyz = np.asarray(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    tri = _orient_outward(xyz, f, np.asarray(center, dtype=np.float64)).astype(np.int32)
    return xyz, tri


def box(lo, hi, divisions):
    """Surface of the axis-aligned box [lo, hi] with a structured triangulation.

    ``divisions`` = (nx, ny, nz) cells along each axis; each surface quad is cut
    into two triangles along alternating diagonals.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = [int(d) for d in divisions]
    index = {}
    verts = []

    def vid(i, j, k):
        key = (i, j, k)
        if key not in index:
            index[key] = len(verts)
            t = np.array([i / n[0], j / n[1], k / n[2]])
            verts.append(lo + (hi - lo) * t)
        return index[key]

    tris = []
    for axis in range(3):
        a1, a2 = [a for a in range(3) if a != axis]
        for side in (0, n[axis]):
            for p in range(n[a1]):
                for q in range(n[a2]):
                    ids = []
                    for dp, dq in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        idx = [0, 0, 0]
                        idx[axis] = side
                        idx[a1] = p + dp
                        idx[a2] = q + dq
                        ids.append(vid(*idx))
                    if (p + q) % 2 == 0:
                        tris += [[ids[0], ids[1], ids[2]], [ids[0], ids[2], ids[3]]]
                    else:
                        tris += [[ids[0], ids[1], ids[3]], [ids[1], ids[2], ids[3]]]
    xyz = np.asarray(verts, dtype=np.float64)
    tri = np.asarray(tris, dtype=np.int64)
    # a box is convex: orient every face away from its centre
    tri = _orient_outward(xyz, tri, 0.5 * (lo + hi)).astype(np.int32)
    return xyz, tri


def torus(major, minor, n_major, n_minor, center=(0.0, 0.0, 0.0)):
    """Ring torus around the z axis with an (n_major x n_minor) quad lattice."""
    u = 2.0 * np.pi * np.arange(n_major) / n_major
    v = 2.0 * np.pi * np.arange(n_minor) / n_minor
    uu, vv = np.meshgrid(u, v, indexing="ij")
    x = (major + minor * np.cos(vv)) * np.cos(uu)
    y = (major + minor * np.cos(vv)) * np.sin(uu)
    z = minor * np.sin(vv)
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) + np.asarray(center)
    tris = []
    for i in range(n_major):
        for j in range(n_minor):
            a = i * n_minor + j
            b = ((i + 1) % n_major) * n_minor + j
            c = ((i + 1) % n_major) * n_minor + (j + 1) % n_minor
            d = i * n_minor + (j + 1) % n_minor
            tris += [[a, b, c], [a, c, d]]
    tri = np.asarray(tris, dtype=np.int64)
    # orient away from the tube centre line
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    c = (v0 + v1 + v2) / 3.0 - np.asarray(center)
    ang = np.arctan2(c[:, 1], c[:, 0])
    core = np.stack([major * np.cos(ang), major * np.sin(ang), np.zeros_like(ang)], 1)
    nrm = np.cross(v1 - v0, v2 - v0)
    flip = np.einsum("ij,ij->i", nrm, c - core) < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    return xyz.astype(np.float64), tri.astype(np.int32)


def merge_meshes(parts):
    """Concatenate several (xyz, tri) meshes; returns (xyz, tri, obj) with obj = part id."""
    xyzs, tris, objs = [], [], []
    off = 0
    for k, (x, t) in enumerate(parts):
        xyzs.append(x)
        tris.append(t + off)
        objs.append(np.full(len(t), k, dtype=np.int32))
        off += len(x)
    return np.concatenate(xyzs), np.concatenate(tris).astype(np.int32), np.concatenate(objs)

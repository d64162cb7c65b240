"""RWG basis functions on pairs of adjacent triangles (Sec. II-A, Eq. EFIEdis).

Reading (the paper only names RWG functions): one basis per interior edge,
edges ordered by (smaller vertex id, larger vertex id).  For edge (a, b), a < b,
T+ is the triangle whose cyclic vertex order contains a -> b and T- the one that
contains b -> a.  With free vertices p+ and p-, edge length l and areas A+-:

    f(r) = l / (2 A+) (r - p+)   on T+,     div f = +l / A+
    f(r) = l / (2 A-) (p- - r)   on T-,     div f = -l / A-

Boundary edges (one triangle) carry no basis; an edge with more than two
triangles, or two triangles traversing it in the same direction, is an error.
"""

import numpy as np


class MeshError(ValueError):
    pass


def triangle_geometry(xyz, tri):
    """Areas, unit normals (right-hand rule) and centroids ((v0 + v1) + v2) / 3."""
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    cr = np.cross(v1 - v0, v2 - v0)
    n2 = np.linalg.norm(cr, axis=1)
    if np.any(n2 <= 0.0):
        raise MeshError("degenerate triangle")
    area = 0.5 * n2
    normal = cr / n2[:, None]
    centroid = ((v0 + v1) + v2) / 3.0
    return area, normal, centroid


def build_rwg(xyz, tri):
    """Return a dict describing the RWG functions of a triangle mesh."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    area, normal, centroid = triangle_geometry(xyz, tri)
    edges = {}
    for t in range(len(tri)):
        for i in range(3):
            u, v = int(tri[t, i]), int(tri[t, (i + 1) % 3])
            key = (u, v) if u < v else (v, u)
            edges.setdefault(key, []).append((t, u < v))
    keys = sorted(edges)
    tp, tm, ea, eb = [], [], [], []
    for key in keys:
        lst = edges[key]
        if len(lst) == 1:
            continue
        if len(lst) != 2:
            raise MeshError("edge shared by more than two triangles")
        (t0, fwd0), (t1, fwd1) = lst
        if fwd0 == fwd1:
            raise MeshError("inconsistent triangle orientation")
        if fwd0:
            tp.append(t0)
            tm.append(t1)
        else:
            tp.append(t1)
            tm.append(t0)
        ea.append(key[0])
        eb.append(key[1])
    tp = np.asarray(tp, dtype=np.int64)
    tm = np.asarray(tm, dtype=np.int64)
    ea = np.asarray(ea, dtype=np.int64)
    eb = np.asarray(eb, dtype=np.int64)

    def free_vertex(t):
        tv = tri[t]
        mask = (tv != ea[:, None]) & (tv != eb[:, None])
        return tv[mask]

    pp = free_vertex(tp)
    pm = free_vertex(tm)
    length = np.linalg.norm(xyz[eb] - xyz[ea], axis=1)
    center = (centroid[tp] + centroid[tm]) * 0.5
    return dict(
        xyz=xyz, tri=tri, area=area, normal=normal, centroid=centroid,
        tp=tp, tm=tm, pp=pp, pm=pm, ea=ea, eb=eb, length=length, center=center,
        n=len(tp),
    )


def basis_on_triangle(rwg, n, sign):
    """(triangle id, free-vertex coordinates, coefficient c, sign) of basis n on T+ or T-.

    On that triangle f(r) = sign * c * (r - p) with c = l / (2 A); div f = sign * 2c.
    """
    if sign > 0:
        t, p = rwg["tp"][n], rwg["xyz"][rwg["pp"][n]]
    else:
        t, p = rwg["tm"][n], rwg["xyz"][rwg["pm"][n]]
    c = rwg["length"][n] / (2.0 * rwg["area"][t])
    return t, p, c, float(sign)


def rwg_arrays(rwg):
    """Per (basis, side) arrays: triangle ids [N,2], free vertices [N,2,3], c [N,2], sign [2]."""
    T = np.stack([rwg["tp"], rwg["tm"]], axis=1)
    P = np.stack([rwg["xyz"][rwg["pp"]], rwg["xyz"][rwg["pm"]]], axis=1)
    C = rwg["length"][:, None] / (2.0 * rwg["area"][T])
    S = np.array([1.0, -1.0])
    return T, P, C, S

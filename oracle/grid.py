"""AIM grid, stencil anchors, moment-matching projection weights and near pairs.

Follows Sec. II-B (Eqs. aimL, aimLFR: projection P onto a regular grid,
interpolation W back) and the statement at the start of Sec. IV that moment
matching equals polynomial interpolation of the kernel.  Readings taken where
the paper is silent:

* Grid: per axis a, N_a nodes, spacing h_a and origin o_a.  Unless given,
  h_a = (hi_a - lo_a) / (N_a - 1 - 2m) and o_a = lo_a - m h_a over the vertex
  bounding box [lo, hi], with margin m = floor((n + 1) / 2) nodes.
* Anchor (first stencil node) of basis n, per axis:
  s_a = floor((c_a - o_a) / h_a - (n - 1) / 2), with c the mean of the two
  triangle centroids.  For even n the middle stencil node is the node nearest
  to c (ties round up).  Stencil = nodes s_a .. s_a + n on every axis.
* Projection weights (moment matching, exact for all monomials of per-axis
  degree <= n):  Lambda_f[u, n] = integral of f_n,f(r) l_u(r) dS with l_u the
  tensor-product Lagrange polynomial of stencil node u, f in {x, y, z}
  components of the RWG function and f = rho using div f.  Galerkin testing
  gives W = P^T.
* Local node index u = i + (n+1) (j + (n+1) k) for node (s_x+i, s_y+j, s_z+k).
* Near region: (m, n) is near iff max_a |s_a(m) - s_a(n)| <= R (Chebyshev
  distance of anchors in grid cells), m = n included.
"""

import numpy as np

from .quadrature import triangle_rule, projection_order, map_points
from .rwg import rwg_arrays


class GridError(ValueError):
    pass


def make_grid(xyz, order, n_nodes, h=None, origin=None):
    """Return dict(n=[Nx,Ny,Nz], h=[3], origin=[3], order, margin)."""
    n_nodes = np.asarray(n_nodes, dtype=np.int64)
    m = (order + 1) // 2
    lo = xyz.min(axis=0)
    hi = xyz.max(axis=0)
    if h is None:
        denom = (n_nodes - 1 - 2 * m).astype(np.float64)
        if np.any(denom <= 0):
            raise GridError("grid too small for the stencil margin")
        h = (hi - lo) / denom
        # an axis along which the mesh is flat takes the largest spacing of the others
        flat = (hi - lo) <= 0
        if np.any(flat) and not np.all(flat):
            h = np.where(flat, h.max(), h)
    h = np.asarray(h, dtype=np.float64)
    if np.any(h <= 0):
        raise GridError("non-positive grid spacing")
    if origin is None:
        origin = lo - m * h
    return dict(n=n_nodes, h=h, origin=np.asarray(origin, dtype=np.float64),
                order=int(order), margin=int(m))


def anchors(grid, centers):
    """Integer stencil start per basis [N, 3]; raises GridError if a stencil leaves the grid."""
    o = grid["order"]
    t = (centers - grid["origin"]) / grid["h"] - (o - 1) / 2.0
    s = np.floor(t).astype(np.int64)
    if np.any(s < 0) or np.any(s + o > grid["n"] - 1):
        raise GridError("stencil outside the grid")
    return s


def lagrange_1d(xi, order):
    """Values of the order+1 Lagrange polynomials on nodes 0..order at local coordinate xi."""
    xi = np.asarray(xi, dtype=np.float64)
    out = np.ones(xi.shape + (order + 1,))
    for i in range(order + 1):
        for m in range(order + 1):
            if m != i:
                out[..., i] *= (xi - m) / float(i - m)
    return out


def stencil_offsets(order):
    """Local offsets (i, j, k) of node u = i + (n+1)(j + (n+1)k), shape [(n+1)^3, 3]."""
    p = order + 1
    u = np.arange(p ** 3)
    return np.stack([u % p, (u // p) % p, u // (p * p)], axis=1)


def projection_weights(rwg, grid, anc):
    """Lambda [N, (n+1)^3, 4] for fields (x, y, z, rho)."""
    o = grid["order"]
    p = o + 1
    bary, w = triangle_rule(projection_order(o))
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    N = rwg["n"]
    lam = np.zeros((N, p ** 3, 4))
    for side in range(2):
        t = T[:, side]
        r = map_points(bary, xyz[tri[t, 0]], xyz[tri[t, 1]], xyz[tri[t, 2]])  # [N,Q,3]
        wq = w[None, :] * area[t][:, None]                                     # [N,Q]
        f = S[side] * C[:, side, None, None] * (r - P[:, side, None, :])        # [N,Q,3]
        div = S[side] * 2.0 * C[:, side]                                        # [N]
        xi = (r - grid["origin"]) / grid["h"] - anc[:, None, :]                # [N,Q,3]
        lx = lagrange_1d(xi[..., 0], o)
        ly = lagrange_1d(xi[..., 1], o)
        lz = lagrange_1d(xi[..., 2], o)
        ell = (lz[..., :, None, None] * ly[..., None, :, None] * lx[..., None, None, :])
        ell = ell.reshape(N, len(w), p ** 3)                                    # [N,Q,U]
        for c in range(3):
            lam[:, :, c] += np.einsum("nq,nq,nqu->nu", wq, f[..., c], ell)
        lam[:, :, 3] += div[:, None] * np.einsum("nq,nqu->nu", wq, ell)
    return lam


def near_pairs(anc, radius):
    """CSR (row_ptr, cols) of the near relation; cols ascending in every row."""
    N = len(anc)
    key_dims = anc.max(axis=0) + 2 * radius + 3
    sh = anc + radius + 1

    def key(a):
        return (a[..., 2] * key_dims[1] + a[..., 1]) * key_dims[0] + a[..., 0]

    k = key(sh)
    order = np.argsort(k, kind="stable")
    ks = k[order]
    rng = np.arange(-radius, radius + 1)
    cols_all = []
    rows_all = []
    for dz in rng:
        for dy in rng:
            for dx in rng:
                kk = key(sh + np.array([dx, dy, dz]))
                lo = np.searchsorted(ks, kk, side="left")
                hi = np.searchsorted(ks, kk, side="right")
                cnt = hi - lo
                if cnt.sum() == 0:
                    continue
                r = np.repeat(np.arange(N), cnt)
                starts = np.repeat(lo, cnt)
                within = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                rows_all.append(r)
                cols_all.append(order[starts + within])
    r = np.concatenate(rows_all)
    c = np.concatenate(cols_all)
    idx = np.lexsort((c, r))
    r, c = r[idx], c[idx]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, c


def project(lam, anc, grid, x, fields=(0, 1, 2, 3)):
    """Grid fields g_f = P_f x on the full grid, shape [F, Nz, Ny, Nx] (Eq. aimLFR, P)."""
    o = grid["order"]
    Nx, Ny, Nz = grid["n"]
    off = stencil_offsets(o)
    g = np.zeros((len(fields), Nz, Ny, Nx), dtype=np.complex128)
    node = anc[:, None, :] + off[None, :, :]                     # [N,U,3]
    for fi, f in enumerate(fields):
        np.add.at(g[fi], (node[..., 2], node[..., 1], node[..., 0]), lam[:, :, f] * x[:, None])
    return g


def interpolate(lam, anc, grid, out, fields=(0, 1, 2, 3)):
    """y_n = sum_f sum_u Lambda_f[u, n] out_f[s_n + u]  (W = P^T)."""
    o = grid["order"]
    off = stencil_offsets(o)
    node = anc[:, None, :] + off[None, :, :]
    y = np.zeros(len(anc), dtype=np.complex128)
    for fi, f in enumerate(fields):
        y += np.einsum("nu,nu->n", lam[:, :, f], out[fi][node[..., 2], node[..., 1], node[..., 0]])
    return y

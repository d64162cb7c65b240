"""AIMx combined-field integral equation for closed PEC bodies (Sec. III-B, Eqs. MFIEout, CFIEout,
CFIEdis, KAIMx, CFIEAIMx; test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this module.

Readings used here (the paper writes the CFIE with n x and n x n x operators
and does not spell out the Galerkin form):

* MFIE on a closed PEC surface with outward unit normal n (triangle vertices
  counter-clockwise about n): n x H_total = J just outside, and the tangential
  jump of the double-layer potential gives n x K[J] -> J / 2 + n x PV K[J], so
      J / 2 - n x PV K[J] = n x H_inc,
  K[X](r) = int grad G(r, r') x X(r') dS' (Eqs. opK, ghgf).  Testing with f_m
  and <f_m, n x v> = -<g_m, v>, g_m = n x f_m, gives
      Z_M = G / 2 + K_g,   (K_g)_mn = <g_m, PV K[f_n]>,   V_M = <f_m, n x H_inc>,
  with G the RWG Gram matrix (the residue term of the principal value).
* CFIE = alpha EFIE + (1 - alpha) eta0 MFIE, alpha = 1/2 by default (the
  paper's Eq. CFIEAIMx weighs the two equally):
      Z_C = alpha Z_E + (1 - alpha) eta0 Z_M,
      V_C = alpha <f, E_inc> + (1 - alpha) eta0 <f, n x H_inc>,
  with this library's EFIE Z_E = j w mu (L^A - k^-2 L^Phi).
* AIMx form of K_g (Eq. KAIMx): K_g,s,NR - K_g,s,P + W_g H_grad P_f, with the
  projection P_f of the vector fields of f_n (as for L^A) and an interpolation
  W_g built from the moments of g_m, Lambda_g[u, m] = int (n x f_m) l_u dS.
  H_grad is zero at d = 0 (the direction r-hat is undefined there; the
  constant of Eq. gH00 multiplies it and drops out).  The static near part
  uses the closed-form gradient potential with its principal value (zero for
  coplanar pairs).
"""

import numpy as np

from .constants import MU0, ETA0
from . import greens
from . import grid as gridmod
from .potentials import tri_potentials
from .quadrature import triangle_rule, map_points, projection_order
from .rwg import rwg_arrays
from .sibc import gram

ALPHA = 0.5
Q_NEAR = 5


def normals(rwg):
    """Unit normals of the triangles (right-hand rule on the vertex order)."""
    xyz, tri = rwg["xyz"], rwg["tri"]
    n = np.cross(xyz[tri[:, 1]] - xyz[tri[:, 0]], xyz[tri[:, 2]] - xyz[tri[:, 0]])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def rotated_weights(rwg, grid, anc):
    """Lambda_g [N, U, 3] = int (n x f_m)_c l_u dS, the rule of the projection weights."""
    o = grid["order"]
    p = o + 1
    bary, w = triangle_rule(projection_order(o))
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    nrm = normals(rwg)
    N = rwg["n"]
    lam = np.zeros((N, p ** 3, 3))
    for side in range(2):
        t = T[:, side]
        r = map_points(bary, xyz[tri[t, 0]], xyz[tri[t, 1]], xyz[tri[t, 2]])
        wq = w[None, :] * area[t][:, None]
        g = np.cross(nrm[t][:, None, :], S[side] * C[:, side, None, None] * (r - P[:, side, None, :]))
        xi = (r - grid["origin"]) / grid["h"] - anc[:, None, :]
        lx = gridmod.lagrange_1d(xi[..., 0], o)
        ly = gridmod.lagrange_1d(xi[..., 1], o)
        lz = gridmod.lagrange_1d(xi[..., 2], o)
        ell = (lz[..., :, None, None] * ly[..., None, :, None] * lx[..., None, None, :]).reshape(N, len(w), p ** 3)
        for c in range(3):
            lam[:, :, c] += np.einsum("nq,nq,nqu->nu", wq, g[..., c], ell)
    return lam


def static_kg(rwg, rows, cols, q=Q_NEAR):
    """(K_g)_s on the pairs: int g_m(r) . [grad_r I1(r) x f_n-part] / (4 pi), principal value."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    nrm = normals(rwg)
    bary, w = triangle_rule(q)
    out = np.zeros(len(rows))
    for so in range(2):
        to = T[rows, so]
        ro = map_points(bary, xyz[tri[to, 0]], xyz[tri[to, 1]], xyz[tri[to, 2]])       # [B, Q, 3]
        wo = w[None, :] * area[to][:, None]
        go = np.cross(nrm[to][:, None, :], S[so] * C[rows, so, None, None] * (ro - P[rows, so, None, :]))
        for ss in range(2):
            ts = T[cols, ss]
            vs = [xyz[tri[ts, i]][:, None, :] for i in range(3)]
            _, _, gI1, _ = tri_potentials(ro, vs[0], vs[1], vs[2])
            kv = (S[ss] * C[cols, ss])[:, None, None] * np.cross(gI1, ro - P[cols, ss][:, None, :])
            out += np.einsum("bq,bqk,bqk->b", wo, go, kv) / (4.0 * np.pi)
    return out


def precorrection_kg(lam, lam_g, anc, grid, rows, cols, radius, chunk=4000):
    """sum_{u,v} Lambda_g[u,m] . (H_s,grad[s_m+u-s_n-v] x Lambda_f[v,n]), grad(1/(4 pi r)), 0 at d = 0."""
    o = grid["order"]
    off = gridmod.stencil_offsets(o)
    span = radius + o
    _, Hg = greens.static_offset_kernels(grid["h"], span)                   # [3, D, D, D]
    duv = off[:, None, :] - off[None, :, :]
    out = np.zeros(len(rows))
    for c0 in range(0, len(rows), chunk):
        m = rows[c0:c0 + chunk]
        n = cols[c0:c0 + chunk]
        d = (anc[m] - anc[n])[:, None, None, :] + duv[None] + span            # [B, U, V, 3]
        idx = (d[..., 2], d[..., 1], d[..., 0])
        hg = np.stack([Hg[a][idx] for a in range(3)], axis=-1)               # [B, U, V, 3]
        cr = np.cross(hg, lam[n][:, None, :, :3])                            # [B, U, V, 3]
        out[c0:c0 + chunk] = np.einsum("buc,buvc->b", lam_g[m], cr)
    return out


def setup_cfie(prob):
    """Adds Lambda_g, the near K_g (static direct - precorrection) and the near Gram matrix to prob."""
    rows, cols = prob["near"]["rows"], prob["cols"]
    lam_g = rotated_weights(prob["rwg"], prob["grid"], prob["anc"])
    kg = static_kg(prob["rwg"], rows, cols) - precorrection_kg(prob["lam"], lam_g, prob["anc"], prob["grid"], rows,
                                                               cols, prob["radius"])
    prob["lam_g"] = lam_g
    prob["near"]["NKG"] = kg
    prob["near"]["G"] = gram(prob["rwg"], rows, cols)
    return prob


def _near(prob, key, x):
    y = np.zeros(prob["N"], dtype=np.complex128)
    np.add.at(y, prob["near"]["rows"], prob["near"][key] * x[prob["cols"]])
    return y


def matvec_mfie(prob, freq, x):
    """Z_M x = G x / 2 + K_g x (AIMx form; grid part by direct summation)."""
    k = 2.0 * np.pi * freq / (ETA0 / MU0)
    g = prob["grid"]
    f = gridmod.project(prob["lam"], prob["anc"], g, x, fields=(0, 1, 2))
    Hg = greens.grad_kernel_table(k, g["n"], g["h"])
    from .operator import cross_conv_full
    out = cross_conv_full(Hg, f)
    node = prob["anc"][:, None, :] + gridmod.stencil_offsets(g["order"])[None]
    idx = (node[..., 2], node[..., 1], node[..., 0])
    kgrid = sum(np.einsum("nu,nu->n", prob["lam_g"][:, :, c], out[c][idx]) for c in range(3))
    return 0.5 * _near(prob, "G", x) + _near(prob, "NKG", x) + kgrid


def matvec_cfie(prob, freq, x, alpha=ALPHA):
    from . import operator as op
    return alpha * op.matvec_efie(prob, freq, x) + (1.0 - alpha) * ETA0 * matvec_mfie(prob, freq, x)


def dense_cfie(prob, freq, alpha=ALPHA):
    """Dense AIMx CFIE matrix, column by column from the product."""
    N = prob["N"]
    from . import operator as op
    ZE = op.dense_efie(prob, freq)
    ZM = np.zeros((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for n in range(N):
        e[:] = 0
        e[n] = 1
        ZM[:, n] = matvec_mfie(prob, freq, e)
    return alpha * ZE + (1.0 - alpha) * ETA0 * ZM


def planewave_rhs_cfie(rwg, k, direction, pol, alpha=ALPHA, e0=1.0):
    """alpha <f, E_inc> + (1 - alpha) eta0 <f, n x H_inc> for a plane wave."""
    from .excitation import tested_field
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(pol, dtype=np.complex128)
    hd = np.cross(d, p) / ETA0
    nrm = normals(rwg)
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(5)
    VE = tested_field(rwg, lambda r: e0 * np.exp(-1j * k * np.einsum("...k,k->...", r, d))[..., None] * p)
    VM = np.zeros(rwg["n"], dtype=np.complex128)
    for side in range(2):
        t = T[:, side]
        r = map_points(bary, xyz[tri[t, 0]], xyz[tri[t, 1]], xyz[tri[t, 2]])
        f = S[side] * C[:, side, None, None] * (r - P[:, side, None, :])
        H = e0 * np.exp(-1j * k * np.einsum("nqk,k->nq", r, d))[..., None] * hd
        nxH = np.cross(nrm[t][:, None, :], H)
        VM += np.einsum("nq,nqk,nqk->n", w[None, :] * area[t][:, None], f, nxH)
    return alpha * VE + (1.0 - alpha) * ETA0 * VM

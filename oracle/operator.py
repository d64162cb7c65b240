"""The AIMx operator by direct (non-FFT) grid summation (Eqs. LAIMx, EFIEAIMx, KAIMx).

A(k) x = N x + W H(k) P x with N = L_s,NR - L_s,P frequency independent
(Eq. LAIMx).  The grid product H g is evaluated here by its definition,
out[u] = sum_v H[u - v] g[v] over all grid nodes v (Eq. Hmn), never by FFT.

Formulations (readings; the paper writes out the EFIE and CFIE for PEC only):

* EFIE for a PEC body in a background (mu, eps), Galerkin RWG testing:
      Z = j w mu [ L^A - k^{-2} L^Phi ],   V_m = <f_m, E_inc>
  (the same system as Eq. EFIEdis up to the overall sign and the sign folded
  into the scalar-potential term, since <f, grad phi> = -<div f, phi>).
* Two-region PMCHWT for a penetrable body (the paper states the method applies
  to penetrable objects; region 1 outside, region 2 inside, unknowns
  x = [J ; M / eta0], equations [E ; eta0 H]):
      y_E = sum_i j w mu_i <L_i> J + eta0 sum_i <K_i> M~
      y_H = -eta0 sum_i <K_i> J + eta0^2 sum_i j w eps_i <L_i> M~
  with <L_i> = L^A_i - k_i^{-2} L^Phi_i and <K_i> = K_i, each taking the AIMx
  form N + W H_i P with the shared static near matrices.
"""

import numpy as np

from .constants import MU0, EPS0, ETA0
from . import grid as gridmod
from . import greens
from . import static as staticmod
from .rwg import build_rwg


# ------------------------------------------------------------------ setup

def setup(xyz, tri, order, n_nodes, radius=3, h=None, origin=None, near_rows=None):
    """Geometry, grid, anchors, weights and near matrices (all rows, or ``near_rows`` only)."""
    rwg = build_rwg(xyz, tri)
    g = gridmod.make_grid(rwg["xyz"], order, n_nodes, h=h, origin=origin)
    anc = gridmod.anchors(g, rwg["center"])
    lam = gridmod.projection_weights(rwg, g, anc)
    row_ptr, cols = gridmod.near_pairs(anc, radius)
    prob = dict(rwg=rwg, grid=g, anc=anc, lam=lam, row_ptr=row_ptr, cols=cols,
                radius=radius, N=rwg["n"])
    if near_rows is None:
        prob["near"] = staticmod.near_matrices(rwg, lam, anc, g, row_ptr, cols, radius)
        prob["near_rows"] = None
    else:
        near_rows = np.asarray(near_rows, dtype=np.int64)
        sub_ptr = np.zeros(len(near_rows) + 1, dtype=np.int64)
        sub_cols = []
        for i, m in enumerate(near_rows):
            c = cols[row_ptr[m]:row_ptr[m + 1]]
            sub_cols.append(c)
            sub_ptr[i + 1] = sub_ptr[i] + len(c)
        sub_cols = np.concatenate(sub_cols)
        rows = np.repeat(near_rows, np.diff(sub_ptr))
        LA, LP, KK = staticmod.static_direct(rwg, rows, sub_cols)
        PA, PP, PK = staticmod.precorrection(lam, anc, g, rows, sub_cols, radius)
        prob["near"] = dict(NA=LA - PA, NP=LP - PP, NK=KK - PK, rows=rows, cols=sub_cols,
                            ptr=sub_ptr, LA=LA, LP=LP, KK=KK)
        prob["near_rows"] = near_rows
    return prob


def near_apply(prob, which, x, rows=None):
    """(N_which x) for all rows, or for ``rows`` when the problem holds sampled near rows."""
    nr = prob["near"]
    vals = nr[which]
    if prob["near_rows"] is None:
        r = nr["rows"]
        y = np.zeros(prob["N"], dtype=np.complex128)
        np.add.at(y, r, vals * x[prob["cols"]])
        return y if rows is None else y[rows]
    ptr = nr["ptr"]
    sel = {int(m): i for i, m in enumerate(prob["near_rows"])}
    y = np.zeros(len(rows), dtype=np.complex128)
    for j, m in enumerate(rows):
        i = sel[int(m)]
        s, e = ptr[i], ptr[i + 1]
        y[j] = np.sum(vals[s:e] * x[nr["cols"][s:e]])
    return y


# ------------------------------------------------------------------ grid products

def conv_full(table, g):
    """out[f, u] = sum_v table[u - v] g[f, v] for every node u (direct summation)."""
    F, Nz, Ny, Nx = g.shape
    out = np.zeros_like(g)
    nz = np.argwhere(np.any(g != 0, axis=0))
    for vz, vy, vx in nz:
        win = table[Nz - 1 - vz:2 * Nz - 1 - vz, Ny - 1 - vy:2 * Ny - 1 - vy,
                    Nx - 1 - vx:2 * Nx - 1 - vx]
        out += g[:, vz, vy, vx, None, None, None] * win[None]
    return out


def conv_nodes(table, g, nodes):
    """out[f, i] = sum_v table[nodes[i] - v] g[f, v] at selected nodes [M,3] (x,y,z)."""
    F, Nz, Ny, Nx = g.shape
    flip = table[::-1, ::-1, ::-1]
    out = np.zeros((F, len(nodes)), dtype=np.complex128)
    gf = g.reshape(F, -1)
    for i, (ux, uy, uz) in enumerate(nodes):
        win = flip[Nz - 1 - uz:2 * Nz - 1 - uz, Ny - 1 - uy:2 * Ny - 1 - uy,
                   Nx - 1 - ux:2 * Nx - 1 - ux]
        out[:, i] = gf @ win.reshape(-1)
    return out


def cross_conv_full(gtab, gvec):
    """out = Hgrad (*) x gvec: out[a] = sum_v (Hgrad[u-v] x gvec[v])_a on the full grid."""
    c = [[conv_full(gtab[a], gvec[b:b + 1])[0] for b in range(3)] for a in range(3)]
    return np.stack([c[1][2] - c[2][1], c[2][0] - c[0][2], c[0][1] - c[1][0]])


def cross_conv_nodes(gtab, gvec, nodes):
    c = [conv_nodes(gtab[a], gvec, nodes) for a in range(3)]  # c[a][b] = Hg_a * g_b
    return np.stack([c[1][2] - c[2][1], c[2][0] - c[0][2], c[0][1] - c[1][0]])


# ------------------------------------------------------------------ operator

def materials(freq, eps_out=1.0, eps_in=None, mu_in=1.0):
    """Angular frequency and per-region (mu, eps, k)."""
    w = 2.0 * np.pi * freq
    regs = [(MU0, EPS0 * eps_out)]
    if eps_in is not None:
        regs.append((MU0 * mu_in, EPS0 * eps_in))
    return w, [(mu, eps, w * np.sqrt(mu * eps)) for mu, eps in regs]


def _grid_parts(prob, k, xs, rows, want_grad):
    """Return per input vector: (GA, GPhi, GK) = (Pv^T H Pv x, Prho^T H Prho x, Pv^T (Hgrad x) Pv x)."""
    g = prob["grid"]
    lam, anc = prob["lam"], prob["anc"]
    H = greens.kernel_table(k, g["n"], g["h"])
    Hg = greens.grad_kernel_table(k, g["n"], g["h"]) if want_grad else None
    off = gridmod.stencil_offsets(g["order"])
    res = []
    for x in xs:
        f = gridmod.project(lam, anc, g, x)
        if rows is None:
            out = conv_full(H, f)
            GA = gridmod.interpolate(lam, anc, g, out[:3], fields=(0, 1, 2))
            GP = gridmod.interpolate(lam, anc, g, out[3:], fields=(3,))
            GK = None
            if want_grad:
                ok = cross_conv_full(Hg, f[:3])
                GK = gridmod.interpolate(lam, anc, g, ok, fields=(0, 1, 2))
        else:
            nodes = (anc[rows][:, None, :] + off[None]).reshape(-1, 3)
            uniq, inv = np.unique(nodes, axis=0, return_inverse=True)
            inv = inv.reshape(len(rows), -1)
            out = conv_nodes(H, f, uniq)
            lr = lam[rows]
            GA = sum(np.einsum("nu,nu->n", lr[:, :, c], out[c][inv]) for c in range(3))
            GP = np.einsum("nu,nu->n", lr[:, :, 3], out[3][inv])
            GK = None
            if want_grad:
                ok = cross_conv_nodes(Hg, f[:3], uniq)
                GK = sum(np.einsum("nu,nu->n", lr[:, :, c], ok[c][inv]) for c in range(3))
        res.append((GA, GP, GK))
    return res


def matvec_efie(prob, freq, x, eps_bg=1.0, rows=None):
    """y = j w mu [ (N^A + Pv^T H Pv) x - k^{-2} (N^Phi + Prho^T H Prho) x ]  (Eq. EFIEAIMx)."""
    w, regs = materials(freq, eps_bg)
    mu, eps, k = regs[0]
    (GA, GP, _), = _grid_parts(prob, k, [x], rows, False)
    NA = near_apply(prob, "NA", x, rows)
    NP = near_apply(prob, "NP", x, rows)
    return 1j * w * mu * ((NA + GA) - (NP + GP) / k ** 2)


def matvec_pmchwt(prob, freq, x, eps_out, eps_in, mu_in=1.0, rows=None):
    """Two-region PMCHWT AIMx product, x = [J ; M/eta0], y = [E-rows ; eta0 H-rows]."""
    N = prob["N"]
    xJ, xM = x[:N], x[N:]
    w, regs = materials(freq, eps_out, eps_in, mu_in)
    nJ = {c: near_apply(prob, c, xJ, rows) for c in ("NA", "NP", "NK")}
    nM = {c: near_apply(prob, c, xM, rows) for c in ("NA", "NP", "NK")}
    yE = 0.0
    yH = 0.0
    for mu, eps, k in regs:
        (GAJ, GPJ, GKJ), (GAM, GPM, GKM) = _grid_parts(prob, k, [xJ, xM], rows, True)
        LJ = (nJ["NA"] + GAJ) - (nJ["NP"] + GPJ) / k ** 2
        LM = (nM["NA"] + GAM) - (nM["NP"] + GPM) / k ** 2
        KJ = nJ["NK"] + GKJ
        KM = nM["NK"] + GKM
        yE = yE + 1j * w * mu * LJ + ETA0 * KM
        yH = yH - ETA0 * KJ + ETA0 ** 2 * 1j * w * eps * LM
    return np.concatenate([yE, yH])


# ------------------------------------------------------------------ dense assembly (small N)

def _grid_matrices(prob, k, want_grad):
    """Dense Pv^T H Pv, Prho^T H Prho and Pv^T (Hgrad x) Pv, built column by column."""
    g = prob["grid"]
    lam, anc = prob["lam"], prob["anc"]
    N = prob["N"]
    Nx, Ny, Nz = g["n"]
    H = greens.kernel_table(k, g["n"], g["h"])
    Hg = greens.grad_kernel_table(k, g["n"], g["h"]) if want_grad else None
    off = gridmod.stencil_offsets(g["order"])
    node = anc[:, None, :] + off[None]
    GA = np.zeros((N, N), dtype=np.complex128)
    GP = np.zeros((N, N), dtype=np.complex128)
    GK = np.zeros((N, N), dtype=np.complex128) if want_grad else None
    idx = (node[..., 2], node[..., 1], node[..., 0])
    for n in range(N):
        out = np.zeros((4, Nz, Ny, Nx), dtype=np.complex128)
        outk = np.zeros((3, Nz, Ny, Nx), dtype=np.complex128) if want_grad else None
        for u in range(len(off)):
            vx, vy, vz = node[n, u]
            sl = (slice(Nz - 1 - vz, 2 * Nz - 1 - vz), slice(Ny - 1 - vy, 2 * Ny - 1 - vy),
                  slice(Nx - 1 - vx, 2 * Nx - 1 - vx))
            win = H[sl]
            out += lam[n, u, :, None, None, None] * win[None]
            if want_grad:
                lv = lam[n, u, :3]
                gw = [Hg[a][sl] for a in range(3)]
                outk[0] += gw[1] * lv[2] - gw[2] * lv[1]
                outk[1] += gw[2] * lv[0] - gw[0] * lv[2]
                outk[2] += gw[0] * lv[1] - gw[1] * lv[0]
        GA[:, n] = sum(np.einsum("mu,mu->m", lam[:, :, c], out[c][idx]) for c in range(3))
        GP[:, n] = np.einsum("mu,mu->m", lam[:, :, 3], out[3][idx])
        if want_grad:
            GK[:, n] = sum(np.einsum("mu,mu->m", lam[:, :, c], outk[c][idx]) for c in range(3))
    return GA, GP, GK


def near_dense(prob, which):
    N = prob["N"]
    A = np.zeros((N, N))
    A[prob["near"]["rows"], prob["cols"]] = prob["near"][which]
    return A


def dense_efie(prob, freq, eps_bg=1.0):
    w, regs = materials(freq, eps_bg)
    mu, eps, k = regs[0]
    GA, GP, _ = _grid_matrices(prob, k, False)
    return 1j * w * mu * ((near_dense(prob, "NA") + GA) - (near_dense(prob, "NP") + GP) / k ** 2)


def dense_pmchwt(prob, freq, eps_out, eps_in, mu_in=1.0):
    w, regs = materials(freq, eps_out, eps_in, mu_in)
    NA, NP, NK = (near_dense(prob, c) for c in ("NA", "NP", "NK"))
    N = prob["N"]
    Z = np.zeros((2 * N, 2 * N), dtype=np.complex128)
    for mu, eps, k in regs:
        GA, GP, GK = _grid_matrices(prob, k, True)
        L = (NA + GA) - (NP + GP) / k ** 2
        K = NK + GK
        Z[:N, :N] += 1j * w * mu * L
        Z[:N, N:] += ETA0 * K
        Z[N:, :N] -= ETA0 * K
        Z[N:, N:] += ETA0 ** 2 * 1j * w * eps * L
    return Z

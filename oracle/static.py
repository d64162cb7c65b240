"""Frequency-independent near-region matrices of AIMx (Eqs. Lmatdecomp2, aimLPs, LAIMx, KAIMx).

For every near pair (m, n) (see ``grid.near_pairs``):

* L^A_s(m,n)  = int int f_m(r) . f_n(r') G_s dS' dS
* L^Phi_s(m,n)= int int div f_m(r) div' f_n(r') G_s dS' dS
* K_s(m,n)    = int f_m(r) . int grad G_s(r, r') x f_n(r') dS' dS   (principal value)

with G_s = 1 / (4 pi R) (Eq. hgfs) and grad G_s = -Rhat / (4 pi R^2) (Eq. ghgfs).
The inner integral over the source triangle is closed form (``potentials``);
the outer one uses the collapsed Gauss-Legendre rule with ``Q_NEAR`` points per
direction.  For an RWG source f_n = sgn c (r' - p):

    int f_n / R dS'            = sgn c [Jrho + (rho - p) I1]
    int grad_r(1/R) x f_n dS'  = sgn c gI1 x (r - p)

The precorrections are the grid approximation of the same static kernel on
the same pairs (Eq. aimLPs):

* L^A_P(m,n)   = sum_{f=x,y,z} sum_{u,v} Lambda_f[u,m] H_s[s_m+u-s_n-v] Lambda_f[v,n]
* L^Phi_P(m,n) = sum_{u,v} Lambda_rho[u,m] H_s[...] Lambda_rho[v,n]
* K_P(m,n)     = sum_{u,v} Lambda_vec[u,m] . (Hsgrad[...] x Lambda_vec[v,n])

and the stored near matrices are N = (static direct) - (precorrection).
"""

import numpy as np

from .quadrature import triangle_rule, map_points
from .potentials import tri_potentials
from .rwg import rwg_arrays
from .grid import stencil_offsets
from .greens import static_offset_kernels

Q_NEAR = 5
FOUR_PI = 4.0 * np.pi


def static_direct(rwg, rows, cols, q=Q_NEAR, chunk=20000):
    """(L^A_s, L^Phi_s, K_s) for the basis pairs (rows[i], cols[i]).

    The closed-form inner potentials are evaluated once per distinct
    (observation triangle, source triangle) pair and then combined into the
    four triangle combinations of every RWG pair.
    """
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    nt = len(tri)
    bary, w = triangle_rule(q)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    npair = len(rows)
    LA = np.zeros(npair)
    LP = np.zeros(npair)
    KK = np.zeros(npair)
    # distinct triangle pairs over all four combinations
    tkeys = np.concatenate([T[rows, so] * nt + T[cols, ss] for so in range(2) for ss in range(2)])
    uniq, inv = np.unique(tkeys, return_inverse=True)
    inv = inv.reshape(4, npair)
    to_u = uniq // nt
    ts_u = uniq % nt
    nu = len(uniq)
    Qn = len(w)
    I1u = np.zeros((nu, Qn))
    Ju = np.zeros((nu, Qn, 3))
    Gu = np.zeros((nu, Qn, 3))
    RHOu = np.zeros((nu, Qn, 3))
    for c0 in range(0, nu, chunk):
        to = to_u[c0:c0 + chunk]
        ts = ts_u[c0:c0 + chunk]
        ro = map_points(bary, xyz[tri[to, 0]], xyz[tri[to, 1]], xyz[tri[to, 2]])
        vs = [xyz[tri[ts, i]][:, None, :] for i in range(3)]
        I1, J, G, rho = tri_potentials(ro, vs[0], vs[1], vs[2])
        I1u[c0:c0 + chunk] = I1
        Ju[c0:c0 + chunk] = J
        Gu[c0:c0 + chunk] = G
        RHOu[c0:c0 + chunk] = rho
    for so in range(2):
        to = T[rows, so]
        ro = map_points(bary, xyz[tri[to, 0]], xyz[tri[to, 1]], xyz[tri[to, 2]])  # [B,Q,3]
        wo = w[None, :] * area[to][:, None]
        fo = S[so] * C[rows, so, None, None] * (ro - P[rows, so, None, :])
        dvo = S[so] * 2.0 * C[rows, so]
        for ss in range(2):
            u = inv[2 * so + ss]
            I1, J, G, rho = I1u[u], Ju[u], Gu[u], RHOu[u]
            cs = S[ss] * C[cols, ss]
            ps = P[cols, ss][:, None, :]
            vecpot = cs[:, None, None] * (J + (rho - ps) * I1[..., None])
            LA += np.einsum("bq,bqk,bqk->b", wo, fo, vecpot) / FOUR_PI
            LP += dvo * S[ss] * 2.0 * C[cols, ss] * np.einsum("bq,bq->b", wo, I1) / FOUR_PI
            kv = cs[:, None, None] * np.cross(G, ro - ps)
            KK += np.einsum("bq,bqk,bqk->b", wo, fo, kv) / FOUR_PI
    return LA, LP, KK


def precorrection(lam, anc, grid, rows, cols, radius, chunk=4000):
    """(L^A_P, L^Phi_P, K_P) on the pairs (rows, cols): grid static kernel between stencils."""
    o = grid["order"]
    off = stencil_offsets(o)
    span = radius + o
    Hs, Hg = static_offset_kernels(grid["h"], span)
    npair = len(rows)
    PA = np.zeros(npair)
    PP = np.zeros(npair)
    PK = np.zeros(npair)
    duv = off[:, None, :] - off[None, :, :]                     # [U,V,3]
    for c0 in range(0, npair, chunk):
        m = rows[c0:c0 + chunk]
        n = cols[c0:c0 + chunk]
        d = (anc[m] - anc[n])[:, None, None, :] + duv[None] + span  # [B,U,V,3]
        idx = (d[..., 2], d[..., 1], d[..., 0])
        hs = Hs[idx]                                                # [B,U,V]
        lm = lam[m]
        ln = lam[n]
        t = hs @ ln                                                 # [B,U,4] = sum_v H_s[u-v] Lambda[v]
        PA[c0:c0 + chunk] = np.einsum("buk,buk->b", lm[:, :, :3], t[:, :, :3])
        PP[c0:c0 + chunk] = np.einsum("bu,bu->b", lm[:, :, 3], t[:, :, 3])
        # sum_{u,v} lm_u . (Hsgrad[u-v] x ln_v), one gradient component b at a time
        tg = [Hg[b][idx] @ ln[:, :, :3] for b in range(3)]          # tg[b][B,U,c]
        acc = np.zeros(len(m))
        for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            acc += np.einsum("bu,bu->b", lm[:, :, a], tg[b][:, :, c])
            acc -= np.einsum("bu,bu->b", lm[:, :, a], tg[c][:, :, b])
        PK[c0:c0 + chunk] = acc
    return PA, PP, PK


def near_matrices(rwg, lam, anc, grid, row_ptr, cols, radius, q=Q_NEAR):
    """Near CSR values N^A, N^Phi, N^K (direct static minus precorrection) and the static diagonal."""
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    LA, LP, KK = static_direct(rwg, rows, cols, q=q)
    PA, PP, PK = precorrection(lam, anc, grid, rows, cols, radius)
    diag = rows == cols
    return dict(NA=LA - PA, NP=LP - PP, NK=KK - PK,
                LsA_diag=LA[diag], LsP_diag=LP[diag], LsK_diag=KK[diag],
                LA=LA, LP=LP, KK=KK, PA=PA, PP=PP, PK=PK, rows=rows)

"""Linear-term accuracy modification of AIMx (Sec. III-A-3, Eqs. linterm and Lmatdecomplin) (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this module.

The Taylor expansion of the Green's function (Eq. hgftaylor) has the term
k^2 G_lin with G_lin(r) = -r / (8 pi) (the (-jk)^2 r / (4 pi 2!) term).  It is
continuous but not smooth at r = 0, so the grid does not reproduce it well
where a basis and a testing function overlap.  The modification integrates it
directly on the overlapping pairs (RWG functions that share a triangle) and
removes the grid's version of it there:

    L += k^2 (L_lin,direct - L_lin,P)   on overlapping pairs,

with L_lin,P the precorrection of the sampled linear kernel
H_lin[d] = -|d h| / (8 pi) between the two stencils (H_lin[0] = 0, the value
of -r / (8 pi) at r = 0).  For the EFIE, Z = j w mu (L^A - k^-2 L^Phi) gains
j w mu (k^2 N^A_lin - N^Phi_lin) x (the k^-2 of the scalar-potential term
cancels the k^2); it is added during the product, scaled by the current k^2.

Direct integrals (the paper does not fix a rule): the inner integral over the
source triangle is in closed form and the outer one uses the 5 x 5 collapsed
Gauss rule of the static near integrals.  With rho the projection of the
observation point r onto the source plane, d its signed height, R = |r - r'|,
and for each edge the quantities of the potentials module (s-, s+, t0, R-, R+,
R0^2 = t0^2 + d^2, f2, outward in-plane normal m), the surface divergence and
gradient theorems give

    div'((rho' - rho) R) = 3 R - d^2 / R   =>   I_R = int_T R dS'
                         = (d^2 I1 + sum_i t0 E1_i) / 3,
    grad'(R^3) = 3 R (rho' - rho)          =>   J_R = int_T (rho' - rho) R dS'
                         = sum_i m_i E3_i / 3,

with the edge integrals E1 = int_e R dl = (s+ R+ - s- R- + R0^2 f2) / 2 and
E3 = int_e R^3 dl = (s+ R+^3 - s- R-^3) / 4 + 3 R0^2 (s+ R+ - s- R-) / 8
+ 3 R0^4 f2 / 8.
"""

import numpy as np

from .grid import stencil_offsets
from .quadrature import triangle_rule, map_points
from .potentials import tri_potentials
from .rwg import rwg_arrays

Q_LIN = 5
EIGHT_PI = 8.0 * np.pi


def r_potentials(r, v0, v1, v2):
    """(I_R, J_R, rho): int_T |r - r'| dS' and int_T (rho' - rho) |r - r'| dS' for a flat triangle T."""
    r, v0, v1, v2 = np.broadcast_arrays(r, v0, v1, v2)
    I1, _, _, rho = tri_potentials(r, v0, v1, v2)
    cr = np.cross(v1 - v0, v2 - v0)
    nrm = cr / np.linalg.norm(cr, axis=-1, keepdims=True)
    d = np.einsum("...k,...k->...", r - v0, nrm)
    IR = d * d * I1
    JR = np.zeros(r.shape)
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        lv = b - a
        lh = lv / np.linalg.norm(lv, axis=-1, keepdims=True)
        mh = np.cross(lh, nrm)
        sm = np.einsum("...k,...k->...", a - rho, lh)
        sp = np.einsum("...k,...k->...", b - rho, lh)
        t0 = np.einsum("...k,...k->...", a - rho, mh)
        Rm = np.linalg.norm(r - a, axis=-1)
        Rp = np.linalg.norm(r - b, axis=-1)
        R02 = t0 * t0 + d * d
        with np.errstate(divide="ignore", invalid="ignore"):
            fa = np.log((Rp + sp) / (Rm + sm))
            fb = np.log((Rm - sm) / (Rp - sp))
        f2 = np.where(sp + sm >= 0.0, fa, fb)
        f2 = np.where(R02 > 0.0, f2, 0.0)                 # R0 = 0: the f2 terms carry a factor R0^2
        E1 = 0.5 * (sp * Rp - sm * Rm + R02 * f2)
        E3 = 0.25 * (sp * Rp ** 3 - sm * Rm ** 3) + 0.375 * R02 * (sp * Rp - sm * Rm) + 0.375 * R02 * R02 * f2
        IR += t0 * E1
        JR += mh * E3[..., None]
    return IR / 3.0, JR / 3.0, rho


def overlapping_pairs(rwg):
    """(rows, cols) of all ordered pairs of RWG functions that share a triangle (m = n included), row-major."""
    T, _, _, _ = rwg_arrays(rwg)
    by_tri = {}
    for m in range(rwg["n"]):
        for t in T[m]:
            by_tri.setdefault(int(t), []).append(m)
    pairs = set()
    for lst in by_tri.values():
        for m in lst:
            for n in lst:
                pairs.add((m, n))
    pairs = sorted(pairs)
    return np.array([p[0] for p in pairs], dtype=np.int64), np.array([p[1] for p in pairs], dtype=np.int64)


def lin_direct(rwg, rows, cols, q=Q_LIN):
    """(L^A_lin, L^Phi_lin): int int (f_m . f_n, div f_m div' f_n) (-R / (8 pi)) over the four triangle pairs."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(q)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    LA = np.zeros(len(rows))
    LP = np.zeros(len(rows))
    for so in range(2):
        to = T[rows, so]
        ro = map_points(bary, xyz[tri[to, 0]], xyz[tri[to, 1]], xyz[tri[to, 2]])      # [B, Q, 3]
        wo = w[None, :] * area[to][:, None]
        fo = S[so] * C[rows, so, None, None] * (ro - P[rows, so, None, :])
        dvo = S[so] * 2.0 * C[rows, so]
        for ss in range(2):
            ts = T[cols, ss]
            vs = [xyz[tri[ts, i]][:, None, :] for i in range(3)]
            IR, JR, rho = r_potentials(ro, vs[0], vs[1], vs[2])
            cs = S[ss] * C[cols, ss]
            vec = cs[:, None, None] * (JR + (rho - P[cols, ss][:, None, :]) * IR[..., None])
            LA -= np.einsum("bq,bqk,bqk->b", wo, fo, vec) / EIGHT_PI
            LP -= dvo * S[ss] * 2.0 * C[cols, ss] * np.einsum("bq,bq->b", wo, IR) / EIGHT_PI
    return LA, LP


def lin_precorrection(lam, anc, grid, rows, cols):
    """(L^A_lin,P, L^Phi_lin,P) = sum_{u,v} Lambda[u,m] H_lin[s_m + u - s_n - v] Lambda[v,n] per component."""
    h = np.asarray(grid["h"], dtype=np.float64)
    off = stencil_offsets(grid["order"])
    PA = np.zeros(len(rows))
    PP = np.zeros(len(rows))
    for k, (m, n) in enumerate(zip(rows, cols)):
        d = (anc[m] - anc[n])[None, None, :] + off[:, None, :] - off[None, :, :]   # [U, V, 3]
        Hl = -np.linalg.norm(d * h, axis=-1) / EIGHT_PI
        t = Hl @ lam[n]                                                             # [U, 4]
        PA[k] = np.sum(lam[m][:, :3] * t[:, :3])
        PP[k] = np.sum(lam[m][:, 3] * t[:, 3])
    return PA, PP


def lin_matrices(prob):
    """Overlapping pairs and N^A_lin, N^Phi_lin = direct - precorrection on them."""
    rows, cols = overlapping_pairs(prob["rwg"])
    LA, LP = lin_direct(prob["rwg"], rows, cols)
    PA, PP = lin_precorrection(prob["lam"], prob["anc"], prob["grid"], rows, cols)
    return rows, cols, LA - PA, LP - PP


def lin_apply(prob, k, x, lin=None):
    """k^2 N^A_lin x and N^Phi_lin x (the two operator parts the modification adds)."""
    rows, cols, NA, NP = lin if lin is not None else lin_matrices(prob)
    a = np.zeros(prob["N"], dtype=np.complex128)
    p = np.zeros(prob["N"], dtype=np.complex128)
    np.add.at(a, rows, k * k * NA * x[cols])
    np.add.at(p, rows, NP * x[cols])
    return a, p


def dense_efie_lin(prob, freq, eps_bg=1.0, lin=None):
    """Dense AIMx EFIE with the linear-term modification."""
    from . import operator as op
    w, regs = op.materials(freq, eps_bg)
    mu, eps, k = regs[0]
    Z = op.dense_efie(prob, freq, eps_bg)
    rows, cols, NA, NP = lin if lin is not None else lin_matrices(prob)
    Z[rows, cols] += 1j * w * mu * (k * k * NA - NP)
    return Z


def matvec_efie_lin(prob, freq, x, eps_bg=1.0, lin=None):
    """AIMx EFIE product with the linear-term modification."""
    from . import operator as op
    w, regs = op.materials(freq, eps_bg)
    mu, eps, k = regs[0]
    a, p = lin_apply(prob, k, x, lin)
    return op.matvec_efie(prob, freq, x, eps_bg) + 1j * w * mu * (a - p)


def matvec_pmchwt_lin(prob, freq, x, eps_out, eps_in, mu_in=1.0, lin=None):
    """Two-region PMCHWT AIMx product with the modification in the L operator of both regions.

    Each region's L = L^A - k^-2 L^Phi gains k^2 N^A_lin - N^Phi_lin, scaled as L
    is in the rows it enters (j w mu on J in the E rows, eta0^2 j w eps on M/eta0
    in the H rows); the K operator is unchanged.
    """
    from . import operator as op
    from .constants import ETA0
    N = prob["N"]
    lin = lin if lin is not None else lin_matrices(prob)
    w, regs = op.materials(freq, eps_out, eps_in, mu_in)
    y = op.matvec_pmchwt(prob, freq, x, eps_out, eps_in, mu_in)
    addE = np.zeros(N, dtype=np.complex128)
    addH = np.zeros(N, dtype=np.complex128)
    for mu, eps, k in regs:
        aJ, pJ = lin_apply(prob, k, x[:N], lin)
        aM, pM = lin_apply(prob, k, x[N:], lin)
        addE += 1j * w * mu * (aJ - pJ)
        addH += ETA0 ** 2 * 1j * w * eps * (aM - pM)
    return y + np.concatenate([addE, addH])

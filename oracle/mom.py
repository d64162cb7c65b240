"""Dense method-of-moments EFIE by direct integration (the error reference, not the parity target).

Every entry of L^A = int int f_m . f_n G and L^Phi = int int div f_m div f_n G
(Eq. EFIEdis) is integrated directly with the paper's split G = G_s + G_d
(Eqs. hgfdecomp0, hgfs, hgfd): the singular G_s part with the closed-form
inner potentials of ``potentials`` and the smooth G_d part with a product
Gauss rule on both triangles.  Z = j w mu (L^A - k^-2 L^Phi).
Feasible for a few thousand unknowns at most.
"""

import numpy as np

from .quadrature import triangle_rule, map_points
from .potentials import tri_potentials
from .rwg import rwg_arrays
from .greens import G_d
from .operator import materials

Q_MOM = 5


def triangle_tables(rwg, k, q=Q_MOM):
    """S0[t, t', i] = int_T' G(r_i, r') dS',  S1[t, t', i] = int_T' r' G(r_i, r') dS' at obs points r_i."""
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    nt = len(tri)
    bary, w = triangle_rule(q)
    pts = map_points(bary, xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]])  # [nt,Q,3]
    wts = w[None, :] * area[:, None]
    Q = len(w)
    S0 = np.zeros((nt, nt, Q), dtype=np.complex128)
    S1 = np.zeros((nt, nt, Q, 3), dtype=np.complex128)
    for t in range(nt):
        r = pts[t][None, :, :]                                        # [1,Q,3]
        v = [xyz[tri[:, i]][:, None, :] for i in range(3)]            # [nt,1,3]
        I1, J, _, rho = tri_potentials(r, v[0], v[1], v[2])           # [nt,Q]
        S0[t] = I1 / (4.0 * np.pi)
        S1[t] = (J + rho * I1[..., None]) / (4.0 * np.pi)
        R = np.linalg.norm(r[:, :, None, :] - pts[:, None, :, :], axis=-1)  # [nt,Q,Q']
        gd = np.where(R > 0, G_d(k, np.where(R > 0, R, 1.0)), -1j * k / (4.0 * np.pi))
        S0[t] += np.einsum("tiq,tq->ti", gd, wts)
        S1[t] += np.einsum("tiq,tq,tqk->tik", gd, wts, pts)
    return pts, wts, S0, S1


def dense_efie_mom(rwg, freq, eps_bg=1.0):
    w_, regs = materials(freq, eps_bg)
    mu, eps, k = regs[0]
    pts, wts, S0, S1 = triangle_tables(rwg, k)
    T, P, C, S = rwg_arrays(rwg)
    N = rwg["n"]
    LA = np.zeros((N, N), dtype=np.complex128)
    LP = np.zeros((N, N), dtype=np.complex128)
    for so in range(2):
        tm = T[:, so]
        fo = S[so] * C[:, so, None, None] * (pts[tm] - P[:, so, None, :])   # [N,Q,3]
        Wo = wts[tm]                                                         # [N,Q]
        dvo = S[so] * 2.0 * C[:, so]
        for ss in range(2):
            tn = T[:, ss]
            s0 = S0[tm][:, tn]                                               # [N,N,Q]
            s1 = S1[tm][:, tn]                                               # [N,N,Q,3]
            pn = P[:, ss]
            cn = S[ss] * C[:, ss]
            vec = s1 - pn[None, :, None, :] * s0[..., None]
            LA += np.einsum("mq,mqk,mnqk->mn", Wo, fo, vec) * cn[None, :]
            LP += np.einsum("mq,mnq->mn", Wo, s0) * (dvo[:, None] * (S[ss] * 2.0 * C[:, ss])[None, :])
    return 1j * w_ * mu * (LA - LP / k ** 2), LA, LP

"""Charge-form scalar potential of the EFIE with AIMx acceleration, by direct grid summation.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline may import
this module.

The EFIE's scalar-potential operator L^Phi_mn = int int div f_m div' f_n G is written through
the charges the currents carry.  With the charge on triangle t as a pulse of density q_t / A_t,
the RWG divergence gives the incidence D_tn = int_{T_t} div f_n dS = +-l_n, and

    L^Phi = D^T Pt D,        Pt_ij = (A_i A_j)^-1 int_{T_i} int_{T_j} G dS' dS

(the discretisation of the augmented EFIE, which the paper cites for electrically small
conductors).  AIMx accelerates Pt exactly as it accelerates the RWG operators (Eq. LAIMx):

    Pt = (Pt_s,NR - Pt_s,P) + Lp^T H(k) Lp

with pulse projection weights Lp[u, t] = A_t^-1 int_{T_t} l_u dS on each triangle's own stencil
(moment matching, Sec. II-B), triangle near pairs by anchor distance, the static kernel
G_s = 1/(4 pi R) for the near part (closed-form inner integral, product rule outside) and its
grid approximation for the precorrection.  The point of the form: a divergence-free current
(D x = 0) gets exactly zero scalar potential whatever the accuracy of the accelerated Pt, while
the RWG form N^Phi + P_rho^T H P_rho leaves an approximation residue on such currents that the
1/k^2 of the EFIE amplifies at small k h.
"""

import numpy as np

from . import greens
from . import grid as gridmod
from .constants import ETA0
from .operator import materials, near_dense, near_apply, conv_full, conv_nodes, _grid_matrices, _grid_parts
from .potentials import tri_potentials
from .quadrature import triangle_rule, map_points, projection_order
from .rwg import rwg_arrays

Q_NEAR = 5
FOUR_PI = 4.0 * np.pi


def incidence(rwg):
    """D [T, N]: D_tn = int_{T_t} div f_n dS = +l_n on T+, -l_n on T-."""
    T, P, C, S = rwg_arrays(rwg)
    D = np.zeros((len(rwg["tri"]), rwg["n"]))
    n = np.arange(rwg["n"])
    np.add.at(D, (T[:, 0], n), rwg["length"])
    np.add.at(D, (T[:, 1], n), -rwg["length"])
    return D


def centroids(rwg):
    return rwg["xyz"][rwg["tri"]].mean(axis=1)


def pulse_weights(rwg, grid, anc_t):
    """Lp [T, (n+1)^3]: A_t^-1 int_{T_t} l_u dS on triangle t's stencil (moments of a unit charge)."""
    o = grid["order"]
    p = o + 1
    bary, w = triangle_rule(projection_order(o))
    xyz, tri = rwg["xyz"], rwg["tri"]
    r = map_points(bary, xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]])   # [T,Q,3]
    xi = (r - grid["origin"]) / grid["h"] - anc_t[:, None, :]
    lx = gridmod.lagrange_1d(xi[..., 0], o)
    ly = gridmod.lagrange_1d(xi[..., 1], o)
    lz = gridmod.lagrange_1d(xi[..., 2], o)
    ell = (lz[..., :, None, None] * ly[..., None, :, None] * lx[..., None, None, :]).reshape(len(tri), len(w), p ** 3)
    return np.einsum("q,tqu->tu", w, ell)           # the area cancels against the 1 / A_t density


def static_pulse(rwg, rows, cols, q=Q_NEAR):
    """Pt_s(i, j) = (A_i A_j)^-1 int_{T_i} int_{T_j} 1/(4 pi R): closed-form inner integral over
    T_j at the q-rule points of T_i."""
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(q)
    ro = map_points(bary, xyz[tri[rows, 0]], xyz[tri[rows, 1]], xyz[tri[rows, 2]])  # [B,Q,3]
    vs = [xyz[tri[cols, i]][:, None, :] for i in range(3)]
    I1 = tri_potentials(ro, vs[0], vs[1], vs[2])[0]                                  # [B,Q]
    return np.einsum("q,bq->b", w, I1) / (FOUR_PI * area[cols])


def pulse_precorrection(Lp, anc_t, grid, rows, cols, radius, chunk=4096):
    """Pt_s,P(i, j) = sum_{u,v} Lp[u, i] H_s[s_i + u - s_j - v] Lp[v, j] on the given pairs
    (evaluated ``chunk`` pairs at a time to bound memory)."""
    o = grid["order"]
    off = gridmod.stencil_offsets(o)
    span = radius + o
    Hs, _ = greens.static_offset_kernels(grid["h"], span)
    out = np.empty(len(rows))
    for a in range(0, len(rows), chunk):
        r, c = rows[a:a + chunk], cols[a:a + chunk]
        d = (anc_t[r] - anc_t[c])[:, None, None, :] + (off[:, None, :] - off[None, :, :])[None] + span
        hs = Hs[(d[..., 2], d[..., 1], d[..., 0])]                                     # [B,U,V]
        out[a:a + chunk] = np.einsum("bu,buv,bv->b", Lp[r], hs, Lp[c])
    return out


def setup_charge(prob, radius=None, tri_rows=None):
    """Triangle anchors, pulse weights, triangle near pairs and the static near values
    N_Pt = Pt_s,NR - Pt_s,P on them, on the grid of an operator problem.  With ``tri_rows``, the
    near values are computed only on the rows of those triangles (NaN elsewhere): enough for
    products restricted to the output rows whose triangles they are."""
    rwg, g = prob["rwg"], prob["grid"]
    radius = prob["radius"] if radius is None else radius
    anc_t = gridmod.anchors(g, centroids(rwg))
    Lp = pulse_weights(rwg, g, anc_t)
    row_ptr, cols = gridmod.near_pairs(anc_t, radius)
    rows = np.repeat(np.arange(len(anc_t)), np.diff(row_ptr))
    sel = np.arange(len(rows)) if tri_rows is None else np.flatnonzero(np.isin(rows, tri_rows))
    Ps = np.full(len(rows), np.nan)
    PP = np.full(len(rows), np.nan)
    Ps[sel] = static_pulse(rwg, rows[sel], cols[sel])
    PP[sel] = pulse_precorrection(Lp, anc_t, g, rows[sel], cols[sel], radius)
    return dict(anc_t=anc_t, Lp=Lp, rows=rows, cols=cols, Ps=Ps, PP=PP, NPt=Ps - PP, D=incidence(rwg),
                radius=radius)


def pt_grid_dense(prob, ch, k):
    """Lp^T H(k) Lp as a dense [T, T] matrix (direct grid summation, column by column)."""
    g = prob["grid"]
    Nx, Ny, Nz = g["n"]
    H = greens.kernel_table(k, g["n"], g["h"])
    off = gridmod.stencil_offsets(g["order"])
    node = ch["anc_t"][:, None, :] + off[None]
    idx = (node[..., 2], node[..., 1], node[..., 0])
    Lp = ch["Lp"]
    nt = len(Lp)
    out = np.zeros((nt, nt), dtype=np.complex128)
    for j in range(nt):
        acc = np.zeros((Nz, Ny, Nx), dtype=np.complex128)
        for u in range(len(off)):
            vx, vy, vz = node[j, u]
            acc += Lp[j, u] * H[Nz - 1 - vz:2 * Nz - 1 - vz, Ny - 1 - vy:2 * Ny - 1 - vy, Nx - 1 - vx:2 * Nx - 1 - vx]
        out[:, j] = np.einsum("iu,iu->i", Lp, acc[idx])
    return out


def pt_dense(prob, ch, k):
    """The AIMx pulse matrix (Pt_s,NR - Pt_s,P) + Lp^T H Lp."""
    nt = len(ch["Lp"])
    N = np.zeros((nt, nt))
    N[ch["rows"], ch["cols"]] = ch["NPt"]
    return N + pt_grid_dense(prob, ch, k)


def lphi_charge_dense(prob, ch, k):
    """L^Phi = D^T Pt D with the AIMx pulse matrix."""
    D = ch["D"]
    return D.T @ pt_dense(prob, ch, k) @ D


def dense_efie_charge(prob, ch, freq, eps_bg=1.0):
    """Z = j w mu [ L^A - k^-2 D^T Pt D ]: the AIMx EFIE with the charge-form scalar potential
    (L^A in the RWG AIMx form, N^A + P_v^T H P_v)."""
    w, regs = materials(freq, eps_bg)
    mu, eps, k = regs[0]
    GA, _, _ = _grid_matrices(prob, k, False)
    LA = near_dense(prob, "NA") + GA
    return 1j * w * mu * (LA - lphi_charge_dense(prob, ch, k) / k ** 2)


def charge_lphi_apply(prob, ch, k, x, rows=None):
    """D^T ((Pt_s,NR - Pt_s,P) + Lp^T H(k) Lp) D x by direct grid summation; with ``rows``, only
    those output rows (the potential is then evaluated on their two triangles only: their stencil
    nodes and their near rows)."""
    g = prob["grid"]
    Nx, Ny, Nz = g["n"]
    H = greens.kernel_table(k, g["n"], g["h"])
    D = ch["D"]
    q = D @ x
    off = gridmod.stencil_offsets(g["order"])
    node = ch["anc_t"][:, None, :] + off[None]
    gq = np.zeros((1, Nz, Ny, Nx), dtype=np.complex128)
    np.add.at(gq[0], (node[..., 2], node[..., 1], node[..., 0]), ch["Lp"] * q[:, None])
    if rows is None:
        tris = np.arange(len(q))
        oq = conv_full(H, gq)[0][node[..., 2], node[..., 1], node[..., 0]]
    else:
        T = rwg_arrays(prob["rwg"])[0]
        tris = np.unique(T[np.asarray(rows)].ravel())
        nodes = node[tris].reshape(-1, 3)
        uniq, inv = np.unique(nodes, axis=0, return_inverse=True)
        oq = conv_nodes(H, gq, uniq)[0][inv.reshape(len(tris), -1)]
    phi = np.zeros(len(q), dtype=np.complex128)
    phi[tris] = np.einsum("tu,tu->t", ch["Lp"][tris], oq)
    sel = np.isin(ch["rows"], tris)
    np.add.at(phi, ch["rows"][sel], ch["NPt"][sel] * q[ch["cols"][sel]])
    LPx = D.T @ phi
    return LPx if rows is None else LPx[np.asarray(rows)]


def matvec_efie_charge(prob, ch, freq, x, eps_bg=1.0, rows=None):
    """y = j w mu [ (N^A + P_v^T H P_v) x - k^-2 D^T ((Pt_s,NR - Pt_s,P) + Lp^T H Lp) D x ]
    by direct grid summation: the charge-form AIMx EFIE product (the RWG form is
    ``operator.matvec_efie``).  With ``rows``, only those output rows."""
    w, regs = materials(freq, eps_bg)
    mu, eps, k = regs[0]
    g = prob["grid"]
    H = greens.kernel_table(k, g["n"], g["h"])
    # vector potential exactly as in the RWG form
    if rows is None:
        f = gridmod.project(prob["lam"], prob["anc"], g, x, fields=(0, 1, 2))
        GA = gridmod.interpolate(prob["lam"], prob["anc"], g, conv_full(H, f), fields=(0, 1, 2))
    else:
        GA = _grid_parts(prob, k, [x], rows, False)[0][0]
    NA = near_apply(prob, "NA", x, rows)
    # scalar potential from the triangle charges q = D x
    LPx = charge_lphi_apply(prob, ch, k, x, rows)
    return 1j * w * mu * ((NA + GA) - LPx / k ** 2)


def dense_pmchwt_charge(prob, ch, freq, eps_out, eps_in, mu_in=1.0):
    """The two-region PMCHWT AIMx matrix (``operator.dense_pmchwt``) with each region's scalar
    potential in charge form, L_r = (N^A + P_v^T H_r P_v) - k_r^-2 D^T Pt(k_r) D, in the J block
    (electric rows) and the M block (magnetic rows) alike; x = [J ; M/eta0]."""
    w, regs = materials(freq, eps_out, eps_in, mu_in)
    NA, NK = near_dense(prob, "NA"), near_dense(prob, "NK")
    N = prob["N"]
    Z = np.zeros((2 * N, 2 * N), dtype=np.complex128)
    for mu, eps, k in regs:
        GA, _, GK = _grid_matrices(prob, k, True)
        L = (NA + GA) - lphi_charge_dense(prob, ch, k) / k ** 2
        K = NK + GK
        Z[:N, :N] += 1j * w * mu * L
        Z[:N, N:] += ETA0 * K
        Z[N:, :N] -= ETA0 * K
        Z[N:, N:] += ETA0 ** 2 * 1j * w * eps * L
    return Z


def matvec_pmchwt_charge(prob, ch, freq, x, eps_out, eps_in, mu_in=1.0, rows=None):
    """The two-region PMCHWT AIMx product (``operator.matvec_pmchwt``) with both regions' scalar
    potentials in charge form, by direct grid summation; x = [J ; M/eta0], y = [E rows ;
    eta0 H rows].  With ``rows`` (indices into 0..N-1), those rows of both blocks."""
    N = prob["N"]
    xJ, xM = x[:N], x[N:]
    w, regs = materials(freq, eps_out, eps_in, mu_in)
    nJ = {c: near_apply(prob, c, xJ, rows) for c in ("NA", "NK")}
    nM = {c: near_apply(prob, c, xM, rows) for c in ("NA", "NK")}
    yE = 0.0
    yH = 0.0
    for mu, eps, k in regs:
        (GAJ, _, GKJ), (GAM, _, GKM) = _grid_parts(prob, k, [xJ, xM], rows, True)
        LJ = (nJ["NA"] + GAJ) - charge_lphi_apply(prob, ch, k, xJ, rows) / k ** 2
        LM = (nM["NA"] + GAM) - charge_lphi_apply(prob, ch, k, xM, rows) / k ** 2
        KJ = nJ["NK"] + GKJ
        KM = nM["NK"] + GKM
        yE = yE + 1j * w * mu * LJ + ETA0 * KM
        yH = yH - ETA0 * KJ + ETA0 ** 2 * 1j * w * eps * LM
    return np.concatenate([yE, yH])

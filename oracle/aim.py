"""Conventional AIM for the EFIE, the comparison method of the paper (Sec. II-B; test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this module.

The conventional AIM splits L(k) = L_NR(k) + L_FR(k) with the far part taken
from the grid and precorrected on the near pairs (Eqs. on L_FR and L_P):

    A(k) x = (L_NR(k) - L_P(k)) x + W H(k) P x,   L_P(k) = W H_NR(k) P,

so both the near-region direct integrals and the precorrection depend on k
and are recomputed at every frequency, where AIMx keeps only static ones.
Readings used here:

* L_NR(k) on a near pair is its full-wave MoM entry: the singular G_s part is
  the static direct integral of ``static`` (closed-form inner potentials, 5 x 5
  outer rule) and the smooth G_d(k) = (e^{-jkR} - 1) / (4 pi R) part uses the
  5 x 5 product rule on both triangles (G_d(0) = -jk / (4 pi)).  This is the
  split and rule of the dense MoM reference, so near entries of AIM equal MoM's.
* L_P(k) samples the same grid kernel H(k) as the FFT product (H[0] is the
  AIMx self-term -jk / (4 pi), Eq. Hmm), so on near pairs the grid's
  contribution cancels exactly.
* EFIE: Z = j w mu [(N^A(k) + P_v^T H P_v) - k^-2 (N^Phi(k) + P_rho^T H P_rho)]
  with N(k) = L_NR(k) - L_P(k) complex.
"""

import numpy as np

from .constants import MU0
from .grid import stencil_offsets
from .quadrature import triangle_rule, map_points
from .rwg import rwg_arrays
from .static import static_direct

Q_DYN = 5


def G_d(k, R):
    """(e^{-jkR} - 1) / (4 pi R) with the limit -jk / (4 pi) at R = 0 (cancellation-free real part)."""
    R = np.asarray(R, dtype=np.float64)
    safe = np.where(R > 0, R, 1.0)
    re = -2.0 * np.sin(0.5 * k * safe) ** 2 / (4.0 * np.pi * safe)
    im = -np.sin(k * safe) / (4.0 * np.pi * safe)
    return np.where(R > 0, re + 1j * im, -1j * k / (4.0 * np.pi))


def dynamic_direct(rwg, rows, cols, k, q=Q_DYN, chunk=2000):
    """(L^A_d, L^Phi_d): int int (f_m . f_n, div f_m div' f_n) G_d(k, R) by the product rule."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    if len(rows) > chunk:
        parts = [dynamic_direct(rwg, rows[c:c + chunk], cols[c:c + chunk], k, q, chunk)
                 for c in range(0, len(rows), chunk)]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(q)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    LA = np.zeros(len(rows), dtype=np.complex128)
    LP = np.zeros(len(rows), dtype=np.complex128)
    for so in range(2):
        to = T[rows, so]
        ro = map_points(bary, xyz[tri[to, 0]], xyz[tri[to, 1]], xyz[tri[to, 2]])       # [B, Q, 3]
        wo = w[None, :] * area[to][:, None]
        fo = S[so] * C[rows, so, None, None] * (ro - P[rows, so, None, :])
        dvo = S[so] * 2.0 * C[rows, so]
        for ss in range(2):
            ts = T[cols, ss]
            rs = map_points(bary, xyz[tri[ts, 0]], xyz[tri[ts, 1]], xyz[tri[ts, 2]])
            ws = w[None, :] * area[ts][:, None]
            fs = S[ss] * C[cols, ss, None, None] * (rs - P[cols, ss, None, :])
            dvs = S[ss] * 2.0 * C[cols, ss]
            R = np.linalg.norm(ro[:, :, None, :] - rs[:, None, :, :], axis=-1)           # [B, Q, Q']
            g = G_d(k, R) * wo[:, :, None] * ws[:, None, :]
            LA += np.einsum("bij,bik,bjk->b", g, fo, fs)
            LP += dvo * dvs * g.sum(axis=(1, 2))
    return LA, LP


def precorrection_k(lam, anc, grid, rows, cols, k):
    """(L^A_P(k), L^Phi_P(k)) = sum_{u,v} Lambda[u,m] H(k)[s_m + u - s_n - v] Lambda[v,n] per component."""
    h = np.asarray(grid["h"], dtype=np.float64)
    off = stencil_offsets(grid["order"])
    PA = np.zeros(len(rows), dtype=np.complex128)
    PP = np.zeros(len(rows), dtype=np.complex128)
    for i, (m, n) in enumerate(zip(rows, cols)):
        d = (anc[m] - anc[n])[None, None, :] + off[:, None, :] - off[None, :, :]
        r = np.linalg.norm(d * h, axis=-1)
        H = np.where(r > 0, np.exp(-1j * k * np.where(r > 0, r, 1.0)) / (4.0 * np.pi * np.where(r > 0, r, 1.0)),
                     -1j * k / (4.0 * np.pi))
        t = H @ lam[n]
        PA[i] = np.sum(lam[m][:, :3] * t[:, :3])
        PP[i] = np.sum(lam[m][:, 3] * t[:, 3])
    return PA, PP


def near_aim(prob, k, static=None):
    """Per-frequency near matrices N^A(k), N^Phi(k) = L_NR(k) - L_P(k) on the near pattern."""
    rows, cols = prob["near"]["rows"], prob["cols"]
    if static is None:
        static = static_direct(prob["rwg"], rows, cols)
    SA, SP = static[0], static[1]
    DA, DP = dynamic_direct(prob["rwg"], rows, cols, k)
    PA, PP = precorrection_k(prob["lam"], prob["anc"], prob["grid"], rows, cols, k)
    return SA + DA - PA, SP + DP - PP


def _materials(freq, eps_bg):
    w = 2.0 * np.pi * freq
    from .constants import EPS0
    eps = EPS0 * eps_bg
    return w, MU0, w * np.sqrt(MU0 * eps)


def matvec_efie_aim(prob, freq, x, eps_bg=1.0, near=None):
    """Conventional-AIM EFIE product (the grid part by direct summation, as in the operator module)."""
    from . import operator as op
    w, mu, k = _materials(freq, eps_bg)
    NA, NP = near if near is not None else near_aim(prob, k)
    rows, cols = prob["near"]["rows"], prob["cols"]
    (GA, GP, _), = op._grid_parts(prob, k, [x], None, False)
    a = np.zeros(prob["N"], dtype=np.complex128)
    p = np.zeros(prob["N"], dtype=np.complex128)
    np.add.at(a, rows, NA * x[cols])
    np.add.at(p, rows, NP * x[cols])
    return 1j * w * mu * ((a + GA) - (p + GP) / k ** 2)


def dense_efie_aim(prob, freq, eps_bg=1.0, near=None):
    """Dense conventional-AIM EFIE matrix."""
    from . import operator as op
    w, mu, k = _materials(freq, eps_bg)
    NA, NP = near if near is not None else near_aim(prob, k)
    GA, GP, _ = op._grid_matrices(prob, k, False)
    rows, cols = prob["near"]["rows"], prob["cols"]
    A = GA.copy()
    Pm = GP.copy()
    A[rows, cols] += NA
    Pm[rows, cols] += NP
    return 1j * w * mu * (A - Pm / k ** 2)

"""Plane-wave right-hand sides <f_m, E_inc> and <f_m, H_inc> (Sec. II-A, Eqs. EFIEdis, CFIEdis).

E_inc(r) = E0 pol exp(-j k d.r)  (e^{j w t}), H_inc = d x E_inc / eta.  The test
integrals use the collapsed Gauss-Legendre rule with ``Q_RHS`` points per
direction on each RWG triangle.
"""

import numpy as np

from .quadrature import triangle_rule, map_points
from .rwg import rwg_arrays

Q_RHS = 5


def tested_field(rwg, field, q=Q_RHS):
    """<f_m, F> for a callable F(points [...,3]) -> [...,3] complex."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(q)
    out = np.zeros(rwg["n"], dtype=np.complex128)
    for side in range(2):
        t = T[:, side]
        r = map_points(bary, xyz[tri[t, 0]], xyz[tri[t, 1]], xyz[tri[t, 2]])
        f = S[side] * C[:, side, None, None] * (r - P[:, side, None, :])
        out += np.einsum("nq,nqk,nqk->n", w[None, :] * area[t][:, None], f, field(r))
    return out


def planewave_rhs(rwg, k, direction, pol, eta=None, e0=1.0):
    """(V_E, V_H) for a plane wave; V_H is None when eta is None."""
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(pol, dtype=np.complex128)

    def E(r):
        ph = np.exp(-1j * k * np.einsum("...k,k->...", r, d))
        return e0 * ph[..., None] * p

    VE = tested_field(rwg, E)
    if eta is None:
        return VE, None
    hd = np.cross(d, p) / eta

    def Hf(r):
        ph = np.exp(-1j * k * np.einsum("...k,k->...", r, d))
        return e0 * ph[..., None] * hd

    return VE, tested_field(rwg, Hf)

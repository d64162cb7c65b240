"""Far field and radar cross section of RWG surface currents (e^{j w t}).

E_far(rhat) r e^{j k r} = -j w mu / (4 pi) int (J - (rhat.J) rhat) e^{j k rhat.r'} dS'
                          + j k / (4 pi) rhat x int M e^{j k rhat.r'} dS'
sigma = 4 pi |E_far|^2 / |E0|^2.
"""

import numpy as np

from .quadrature import triangle_rule, map_points
from .rwg import rwg_arrays

Q_FAR = 5


def radiation_integral(rwg, coef, k, dirs, q=Q_FAR):
    """int sum_n coef_n f_n(r') exp(j k rhat.r') dS' for each rhat in dirs [D,3] -> [D,3]."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri, area = rwg["xyz"], rwg["tri"], rwg["area"]
    bary, w = triangle_rule(q)
    out = np.zeros((len(dirs), 3), dtype=np.complex128)
    for side in range(2):
        t = T[:, side]
        r = map_points(bary, xyz[tri[t, 0]], xyz[tri[t, 1]], xyz[tri[t, 2]])  # [N,Q,3]
        f = S[side] * C[:, side, None, None] * (r - P[:, side, None, :])
        wq = w[None, :] * area[t][:, None]
        ph = np.exp(1j * k * np.einsum("nqk,dk->dnq", r, dirs))             # [D,N,Q]
        out += np.einsum("dnq,nq,n,nqk->dk", ph, wq, coef, f)
    return out


def far_field(rwg, J, k, omega, mu, dirs, M=None):
    dirs = np.asarray(dirs, dtype=np.float64)
    IJ = radiation_integral(rwg, J, k, dirs)
    tang = IJ - np.einsum("dk,dk->d", dirs, IJ)[:, None] * dirs
    E = -1j * omega * mu / (4.0 * np.pi) * tang
    if M is not None:
        IM = radiation_integral(rwg, M, k, dirs)
        E = E + 1j * k / (4.0 * np.pi) * np.cross(dirs, IM)
    return E


def rcs(E, e0=1.0):
    return 4.0 * np.pi * np.sum(np.abs(E) ** 2, axis=-1) / abs(e0) ** 2

"""Closed-form static potentials of a flat triangle (kernel 1/r of Eq. hgfs, grad of Eq. ghgfs).

For an observation point r and a source triangle T (vertices counter-clockwise
about its unit normal n) this module returns

    I1(r)   = integral over T of 1 / |r - r'| dS'
    Jrho(r) = integral over T of (r' - rho) / |r - r'| dS'   (rho = projection of r on T's plane)
    gI1(r)  = grad_r I1(r) = -integral over T of (r - r') / |r - r'|^3 dS'

using the standard edge-sum closed forms for the potential integrals of a
triangle (written out here from the surface divergence theorem):
with d = n.(r - v0), and for each edge i (endpoints a -> b, unit vector l,
outward in-plane normal m = l x n):

    s- = (a - rho).l,  s+ = (b - rho).l,  t0 = (a - rho).m,
    R- = |r - a|, R+ = |r - b|, R0^2 = t0^2 + d^2,
    f2 = ln((R+ + s+) / (R- + s-))         [= ln((R- - s-) / (R+ - s+)) used when s+ + s- < 0]
    beta = atan2(t0 s+, R0^2 + |d| R+) - atan2(t0 s-, R0^2 + |d| R-)

    I1   = sum_i t0 f2 - |d| sum_i beta
    Jrho = 1/2 sum_i m [R0^2 f2 + s+ R+ - s- R-]
    gI1  = -sum_i m f2 - n sgn(d) sum_i beta

sgn(d) is taken as 0 when |d| <= 1e-12 times the longest edge of T, which
gives the principal value on the triangle's plane.
"""

import numpy as np


def tri_potentials(r, v0, v1, v2):
    """Vectorised potentials; r, v0, v1, v2 broadcast to [..., 3]."""
    r, v0, v1, v2 = np.broadcast_arrays(r, v0, v1, v2)
    e1 = v1 - v0
    e2 = v2 - v0
    cr = np.cross(e1, e2)
    nrm = cr / np.linalg.norm(cr, axis=-1, keepdims=True)
    d = np.einsum("...k,...k->...", r - v0, nrm)
    rho = r - d[..., None] * nrm
    ad = np.abs(d)
    scale = np.maximum(np.maximum(np.linalg.norm(e1, axis=-1), np.linalg.norm(e2, axis=-1)),
                       np.linalg.norm(v2 - v1, axis=-1))
    sgn = np.where(ad <= 1e-12 * scale, 0.0, np.sign(d))
    I1 = np.zeros(d.shape)
    J = np.zeros(r.shape)
    G = np.zeros(r.shape)
    bsum = np.zeros(d.shape)
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        lv = b - a
        L = np.linalg.norm(lv, axis=-1, keepdims=True)
        lh = lv / L
        mh = np.cross(lh, nrm)
        sm = np.einsum("...k,...k->...", a - rho, lh)
        sp = np.einsum("...k,...k->...", b - rho, lh)
        t0 = np.einsum("...k,...k->...", a - rho, mh)
        Rm = np.linalg.norm(r - a, axis=-1)
        Rp = np.linalg.norm(r - b, axis=-1)
        R02 = t0 * t0 + d * d
        pos = (sp + sm) >= 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            fa = np.log((Rp + sp) / (Rm + sm))
            fb = np.log((Rm - sm) / (Rp - sp))
        f2 = np.where(pos, fa, fb)
        beta = np.arctan2(t0 * sp, R02 + ad * Rp) - np.arctan2(t0 * sm, R02 + ad * Rm)
        I1 += t0 * f2
        bsum += beta
        J += 0.5 * mh * (R02 * f2 + sp * Rp - sm * Rm)[..., None]
        G -= mh * f2[..., None]
    I1 -= ad * bsum
    G -= nrm * (sgn * bsum)[..., None]
    return I1, J, G, rho

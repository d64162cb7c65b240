"""Collapsed (Duffy) Gauss-Legendre product rule on a triangle.

The paper fixes no quadrature.  Reading: map the unit square to the triangle by
barycentric coordinates (l1, l2, l3) = (u, (1-u) v, (1-u)(1-v)) with Jacobian
proportional to (1-u), and take q Gauss-Legendre points in u and in v.  The rule
integrates every polynomial of total degree <= 2q - 2 exactly.  Weights are
normalised to sum to one (multiply by the triangle area).  Point order: u-index
outer, v-index inner.
"""

import numpy as np


def gauss_legendre01(q):
    """Gauss-Legendre nodes and weights on [0, 1] (library primitive)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(q):
    """Barycentric points [q*q, 3] and normalised weights [q*q]."""
    u, wu = gauss_legendre01(q)
    pts, wts = [], []
    for i in range(q):
        for j in range(q):
            l1 = u[i]
            l2 = (1.0 - u[i]) * u[j]
            l3 = (1.0 - u[i]) * (1.0 - u[j])
            pts.append((l1, l2, l3))
            wts.append(2.0 * wu[i] * wu[j] * (1.0 - u[i]))
    return np.asarray(pts), np.asarray(wts)


def map_points(bary, v0, v1, v2):
    """Cartesian points for barycentric ``bary`` [Q,3] on triangles v* [...,3] -> [...,Q,3]."""
    return (bary[:, 0, None] * v0[..., None, :] + bary[:, 1, None] * v1[..., None, :]
            + bary[:, 2, None] * v2[..., None, :])


def projection_order(order):
    """Points per direction that make the projection moments exact for stencil order n.

    The integrand is an RWG component (degree 1) times a tensor Lagrange
    polynomial of degree n per axis (total degree <= 3n), so q >= (3n + 3) / 2.
    """
    return (3 * order + 4) // 2

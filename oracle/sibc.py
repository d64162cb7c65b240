"""Surface impedance and delta-gap ports for conductors (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this module.

The paper models skin effect with the surface impedance boundary condition and
excites structures with delta-gap ports (Sec. VI), citing both without writing
them out.  Readings used here:

* SIBC (Leontovich): on a good conductor the total tangential field satisfies
  E_tan = Z_s J with Z_s = (1 + j) / (sigma delta), delta = sqrt(2 / (w mu sigma)).
  Galerkin testing of E_inc + E_scat = Z_s J with the EFIE convention of the
  operator module (Z J = <f, E_inc> with Z = j w mu [L^A - k^-2 L^Phi]) gives
  (Z + Z_s G) J = V, where G_mn = int f_m . f_n dS is the RWG Gram matrix
  (non-zero only for bases that share a triangle).  Z_s multiplies a static,
  frequency-independent matrix, so it joins the AIMx near part unchanged in form.
* Delta-gap port: a plane (point r0, unit normal n) cutting a conductor along
  mesh edges; the gap edges are the interior edges lying in the plane whose
  midpoint is inside the port's box.  A voltage V across the gap is the field
  V delta(n.(r - r0)) n, whose test integral is <f_m, E> = V l_m s_m with
  s_m = sign((c_m- - c_m+) . n) (an RWG function carries unit normal flux
  across its own edge, from T+ to T-).  The port current of coefficients x is
  the flux across the same edges, I = sum_m x_m l_m s_m.  Y_ij is the current at
  port i for 1 V at port j and 0 V elsewhere.
"""

import numpy as np

from .constants import MU0
from .quadrature import triangle_rule, map_points
from .rwg import rwg_arrays


def surface_impedance(freq, sigma, mu=MU0):
    """Z_s = (1 + j) / (sigma delta), delta = sqrt(2 / (w mu sigma))."""
    w = 2.0 * np.pi * freq
    delta = np.sqrt(2.0 / (w * mu * sigma))
    return (1.0 + 1.0j) / (sigma * delta)


def gram(rwg, rows, cols, q=3):
    """G_mn = int f_m . f_n dS for the given pairs (degree-2 integrand; the rule is exact)."""
    T, P, C, S = rwg_arrays(rwg)
    xyz, tri = rwg["xyz"], rwg["tri"]
    bary, w = triangle_rule(q)
    out = np.zeros(len(rows))
    for k, (m, n) in enumerate(zip(rows, cols)):
        acc = 0.0
        for a in range(2):
            for b in range(2):
                t = T[m, a]
                if t != T[n, b]:
                    continue
                v = xyz[tri[t]]
                pts = map_points(bary, v[0], v[1], v[2])
                fm = S[a] * C[m, a] * (pts - P[m, a])
                fn = S[b] * C[n, b] * (pts - P[n, b])
                acc += rwg["area"][t] * np.sum(w * np.sum(fm * fn, axis=1))
        out[k] = acc
    return out


def gram_dense(rwg):
    """Dense Gram matrix (all pairs that share a triangle)."""
    N = rwg["n"]
    T, _, _, _ = rwg_arrays(rwg)
    rows, cols = [], []
    by_tri = {}
    for m in range(N):
        for t in T[m]:
            by_tri.setdefault(int(t), []).append(m)
    pairs = set()
    for lst in by_tri.values():
        for m in lst:
            for n in lst:
                pairs.add((m, n))
    pairs = sorted(pairs)
    rows = np.array([p[0] for p in pairs])
    cols = np.array([p[1] for p in pairs])
    G = np.zeros((N, N))
    G[rows, cols] = gram(rwg, rows, cols)
    return G


def port_edges(rwg, point, normal, box_lo, box_hi, tol=1e-9):
    """(basis ids, signs) of the gap edges of a delta-gap port."""
    xyz = rwg["xyz"]
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    p0 = np.asarray(point, dtype=np.float64)
    scale = np.max(rwg["length"])
    da = (xyz[rwg["ea"]] - p0) @ n
    db = (xyz[rwg["eb"]] - p0) @ n
    mid = 0.5 * (xyz[rwg["ea"]] + xyz[rwg["eb"]])
    inside = np.all((mid >= np.asarray(box_lo) - tol * scale) & (mid <= np.asarray(box_hi) + tol * scale), axis=1)
    on = (np.abs(da) <= tol * scale) & (np.abs(db) <= tol * scale) & inside
    ids = np.nonzero(on)[0]
    c = rwg["centroid"]
    s = np.sign((c[rwg["tm"][ids]] - c[rwg["tp"][ids]]) @ n)
    return ids, s


def port_vector(rwg, port):
    """The port's excitation / current functional c with c_m = l_m s_m on its gap edges."""
    ids, s = port_edges(rwg, *port)
    c = np.zeros(rwg["n"])
    c[ids] = rwg["length"][ids] * s
    return c


def y_parameters(Z, rwg, ports):
    """Y [P, P] from the dense system matrix Z: solve Z x_j = c_j, Y_ij = c_i . x_j."""
    Cm = np.stack([port_vector(rwg, p) for p in ports], axis=1)     # [N, P]
    X = np.linalg.solve(Z, Cm.astype(np.complex128))
    return Cm.T @ X


def matvec_efie_sibc(prob, freq, x, sigma, eps_bg=1.0):
    """(Z + Z_s G) x with Z the AIMx EFIE product of the operator module."""
    from . import operator as op
    G = gram(prob["rwg"], prob["near"]["rows"], prob["cols"])
    g = np.zeros(prob["N"], dtype=np.complex128)
    np.add.at(g, prob["near"]["rows"], G * x[prob["cols"]])
    return op.matvec_efie(prob, freq, x, eps_bg) + surface_impedance(freq, sigma) * g


def dense_efie_sibc(prob, freq, sigma, eps_bg=1.0):
    """Dense Z + Z_s G (AIMx EFIE plus the surface-impedance Gram term)."""
    from . import operator as op
    return op.dense_efie(prob, freq, eps_bg) + surface_impedance(freq, sigma) * gram_dense(prob["rwg"])

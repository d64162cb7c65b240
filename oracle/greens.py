"""Green's functions, AIM grid kernels and the Lagrange interpolation error bound.

* G(k, r)     = exp(-j k r) / (4 pi r)                      (Eq. hgf, time convention e^{j w t})
* G_s(r)      = 1 / (4 pi r)                                (Eq. hgfs)
* G_d(k, r)   = (exp(-j k r) - 1) / (4 pi r)                (Eq. hgfd)
* grad G      = -rhat (1 + j k r) exp(-j k r) / (4 pi r^2)  (Eq. ghgf), gradient w.r.t. the
                observation point, rhat = (r - r') / |r - r'|
* grad G_s    = -rhat / (4 pi r^2)                          (Eq. ghgfs)

Grid kernels (first row of the 3-level Toeplitz H, Eq. Hmn) on offsets
d = (dx, dy, dz) with physical separation r_d = (dx hx, dy hy, dz hz):

* H[d]      = G(k, |r_d|),  H[0] = -j k / (4 pi)         (Eqs. Hsmm, Hdmm, Hmm)
* H_s[d]    = G_s(|r_d|),   H_s[0] = 0                    (Eq. Hsmm)
* Hgrad[d]  = grad G at r_d, Hgrad[0] = 0 per component.  Reading: Eq. gH00
  gives only the scalar (-jk)^2 / (8 pi) multiplying the undefined direction
  rhat at r = 0; each Cartesian component is odd in its own offset, so the
  zero-offset sample is taken as 0.
* Hsgrad[d] = grad G_s at r_d, Hsgrad[0] = 0.

The interpolation bound of Sec. IV-A (Eqs. Lbounds, Dhgf, Dghgf) is also here.
"""

import math

import numpy as np


def G(k, r):
    return np.exp(-1j * k * r) / (4.0 * np.pi * r)


def G_s(r):
    return 1.0 / (4.0 * np.pi * r)


def G_d(k, r):
    return (np.exp(-1j * k * r) - 1.0) / (4.0 * np.pi * r)


def offset_vectors(n, h):
    """Physical separations for all offsets d in [-(N-1), N-1]^3: array [2Nz-1, 2Ny-1, 2Nx-1, 3]."""
    ax = [np.arange(-(n[a] - 1), n[a]) * h[a] for a in range(3)]
    dz, dy, dx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([dx, dy, dz], axis=-1)


def kernel_table(k, n, h):
    """H[d] over all offsets (scalar kernel of Eq. Hmn with the AIMx self-term Eq. Hmm)."""
    rv = offset_vectors(n, h)
    r = np.linalg.norm(rv, axis=-1)
    c = tuple(n[a] - 1 for a in (2, 1, 0))
    r[c] = 1.0
    H = G(k, r)
    H[c] = -1j * k / (4.0 * np.pi)
    return H


def grad_kernel_table(k, n, h):
    """Hgrad[d] components [3, ...] (grad G at r_d; zero at d = 0)."""
    rv = offset_vectors(n, h)
    r = np.linalg.norm(rv, axis=-1)
    c = tuple(n[a] - 1 for a in (2, 1, 0))
    r[c] = 1.0
    fac = -(1.0 + 1j * k * r) * np.exp(-1j * k * r) / (4.0 * np.pi * r ** 3)
    out = np.stack([fac * rv[..., a] for a in range(3)])
    out[(slice(None),) + c] = 0.0
    return out


def static_offset_kernels(h, span):
    """H_s and Hsgrad on offsets d in [-span, span]^3 (index d + span), for precorrection."""
    ax = np.arange(-span, span + 1)
    dz, dy, dx = np.meshgrid(ax, ax, ax, indexing="ij")
    rv = np.stack([dx * h[0], dy * h[1], dz * h[2]], axis=-1)
    r = np.linalg.norm(rv, axis=-1)
    c = (span, span, span)
    r[c] = 1.0
    Hs = 1.0 / (4.0 * np.pi * r)
    Hs[c] = 0.0
    Hg = -rv / (4.0 * np.pi * r[..., None] ** 3)
    Hg[c] = 0.0
    return Hs, np.moveaxis(Hg, -1, 0)


# ---------------------------------------------------------------- Sec. IV-A error bound

def dn_Gd(n, theta):
    """(n+1)-th derivative of G_d in normalised distance theta = k r (Eq. Dhgf), k = 1 units.

    Reading: Eq. Dhgf as printed carries (-j theta)^l inside the sum; term-by-term
    differentiation of (e^{-j theta} - 1) / (4 pi theta) gives (+j theta)^l, which
    is what is used here (the symbolic check in the tests pins it).
    """
    m = n + 1
    s = 0.0 + 0.0j
    for l in range(m + 1):
        s += math.comb(m, l) * math.factorial(m - l) / math.factorial(m) * (1j * theta) ** l
    s = -1.0 + s * np.exp(-1j * theta)
    return (-1.0) ** m / (4.0 * np.pi * theta ** (n + 2)) * math.factorial(m) * s


def _pochhammer(a, b):
    out = 1.0
    for i in range(b):
        out *= a + i
    return out


def dn_gradGd(n, theta):
    """(n+1)-th derivative of the radial factor of grad G_d (Eq. Dghgf), without -theta_hat."""
    m = n + 1
    s = 0.0 + 0.0j
    for l in range(m + 1):
        delta = 1.0 if l == 0 else 0.0
        s += (math.comb(m, l) * _pochhammer(-n - 2 + l, m - l) / theta ** (n + 3 - l)
              * (-delta + (-1j) ** l * np.exp(-1j * theta) * (1.0 + 1j * theta - l)))
    return s / (4.0 * np.pi)


def gd_radial(theta):
    """G_d in normalised units (k = 1)."""
    return (np.exp(-1j * theta) - 1.0) / (4.0 * np.pi * theta)


def gradgd_radial(theta):
    """Radial factor F of grad G_d = -rhat F (k = 1):  F = ((1 + j t) e^{-j t} - 1) / (4 pi t^2)."""
    return ((1.0 + 1j * theta) * np.exp(-1j * theta) - 1.0) / (4.0 * np.pi * theta ** 2)


def lagrange_interp_error(func, nodes, theta):
    """|func(theta) - p_n(theta)| for the Lagrange interpolant through ``nodes`` (Sec. IV-A)."""
    vals = func(np.asarray(nodes))
    p = np.zeros(np.shape(theta), dtype=np.complex128)
    for q, tq in enumerate(nodes):
        ell = np.ones(np.shape(theta))
        for m, tm in enumerate(nodes):
            if m != q:
                ell = ell * (theta - tm) / (tq - tm)
        p = p + vals[q] * ell
    return np.abs(func(theta) - p)


def interp_bound(dfunc, n, t0, tn, samples=2000):
    """B_n = (tn - t0)^{n+1} / (n+1)! * max |d^{n+1} K / dtheta^{n+1}| over [t0, tn] (Eq. Lbounds)."""
    xs = np.linspace(t0, tn, samples)
    mx = np.max(np.abs(np.array([dfunc(n, x) for x in xs])))
    return (tn - t0) ** (n + 1) / math.factorial(n + 1) * mx

"""Mie series for a sphere (textbook closed form; independent physics check).

Bistatic RCS for a plane wave travelling along +z with x-polarised E, observed
at polar angle theta in the plane of azimuth phi:

    sigma = 4 pi / k^2 (|S2(theta)|^2 cos^2 phi + |S1(theta)|^2 sin^2 phi)

with S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),
     S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
Riccati-Bessel psi_n(x) = x j_n(x), xi_n(x) = x h_n(x) (spherical Bessel
functions from scipy.special as a library primitive) and

    PEC:          a_n = psi_n'(x) / xi_n'(x),      b_n = psi_n(x) / xi_n(x)
    dielectric:   a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)]
                        / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
                  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)]
                        / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)]

(non-magnetic sphere, relative index m = sqrt(eps_r)).  Magnitudes do not
depend on the time convention.
"""

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, x):
    return x * spherical_jn(n, x), spherical_jn(n, x) + x * spherical_jn(n, x, derivative=True)


def _xi(n, x):
    h = spherical_jn(n, x) + 1j * spherical_yn(n, x)
    dh = spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True)
    return x * h, h + x * dh


def coefficients(x, eps_r=None, nmax=None):
    if nmax is None:
        nmax = int(x + 4.05 * x ** (1.0 / 3.0) + 10)
    n = np.arange(1, nmax + 1)
    ps, dps = _psi(n, x)
    xi, dxi = _xi(n, x)
    if eps_r is None:
        return n, dps / dxi, ps / xi
    m = np.sqrt(eps_r)
    pm, dpm = _psi(n, m * x)
    a = (m * pm * dps - ps * dpm) / (m * pm * dxi - xi * dpm)
    b = (pm * dps - m * ps * dpm) / (pm * dxi - m * xi * dpm)
    return n, a, b


def amplitudes(x, theta, eps_r=None):
    n, a, b = coefficients(x, eps_r)
    mu = np.cos(theta)
    pi = np.zeros((len(n) + 1,) + np.shape(theta))
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    tau[1] = mu
    for i in range(2, len(n) + 1):
        pi[i] = (2 * i - 1) / (i - 1) * mu * pi[i - 1] - i / (i - 1) * pi[i - 2]
        tau[i] = i * mu * pi[i] - (i + 1) * pi[i - 1]
    c = (2 * n + 1) / (n * (n + 1.0))
    S1 = np.tensordot(c * a, pi[1:], axes=1) + np.tensordot(c * b, tau[1:], axes=1)
    S2 = np.tensordot(c * a, tau[1:], axes=1) + np.tensordot(c * b, pi[1:], axes=1)
    return S1, S2


def bistatic_rcs(k, radius, theta, phi, eps_r=None):
    S1, S2 = amplitudes(k * radius, theta, eps_r)
    return 4.0 * np.pi / k ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2
                                   + np.abs(S1) ** 2 * np.sin(phi) ** 2)

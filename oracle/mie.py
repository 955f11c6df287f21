"""Mie series for homogeneous and coated spheres (oracle, test infrastructure).

The paper validates its method against the Mie series (Sect. "Simulation
Results", Fig. 5 two-layer sphere; Fig. 10 coated nanoparticle).  This is the
textbook Lorenz-Mie solution (Bohren & Huffman, Ch. 4) and its Aden-Kerker
extension to a coated sphere (Bohren & Huffman, Sect. 8.1), written from the
formulas with Riccati-Bessel functions psi_n = z j_n, chi_n = -z y_n,
xi_n = psi_n - i chi_n.  The series uses the e^{-i w t} convention of that text;
|S|^2, hence the RCS, does not depend on the convention (indices are conjugated
on input).  Truncation n_max = x + 4 x^{1/3} + 2 (Wiscombe).

Bistatic RCS (incidence along the z axis, x-polarised):
  E-plane (phi = 0):   sigma = (lambda^2 / pi) |S2(Theta)|^2
  H-plane (phi = 90):  sigma = (lambda^2 / pi) |S1(Theta)|^2
Theta is the scattering angle from the forward direction.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    j = spherical_jn(n, z)
    dj = spherical_jn(n, z, derivative=True)
    return z * j, j + z * dj


def _chi(n, z):
    y = spherical_yn(n, z)
    dy = spherical_yn(n, z, derivative=True)
    return -z * y, -(y + z * dy)


def coefficients_homogeneous(x, m, nmax=None):
    if nmax is None:
        nmax = int(np.ceil(abs(x) + 4.0 * abs(x) ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    px, dpx = _psi(n, x)
    cx, dcx = _chi(n, x)
    xi, dxi = px - 1j * cx, dpx - 1j * dcx
    pm, dpm = _psi(n, m * x)
    a = (m * pm * dpx - px * dpm) / (m * pm * dxi - xi * dpm)
    b = (pm * dpx - m * px * dpm) / (pm * dxi - m * xi * dpm)
    return a, b


def coefficients_coated(x, y, m1, m2, nmax=None):
    """Core size parameter x = k a, m1; coating y = k b, m2 (relative indices)."""
    if nmax is None:
        nmax = int(np.ceil(abs(y) + 4.0 * abs(y) ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    p1, dp1 = _psi(n, m1 * x)
    p2x, dp2x = _psi(n, m2 * x)
    c2x, dc2x = _chi(n, m2 * x)
    p2y, dp2y = _psi(n, m2 * y)
    c2y, dc2y = _chi(n, m2 * y)
    py, dpy = _psi(n, y)
    cy, dcy = _chi(n, y)
    xy, dxy = py - 1j * cy, dpy - 1j * dcy
    A = (m2 * p2x * dp1 - m1 * dp2x * p1) / (m2 * c2x * dp1 - m1 * dc2x * p1)
    B = (m2 * p1 * dp2x - m1 * p2x * dp1) / (m2 * dc2x * p1 - m1 * dp1 * c2x)
    a = (py * (dp2y - A * dc2y) - m2 * dpy * (p2y - A * c2y)) / \
        (xy * (dp2y - A * dc2y) - m2 * dxy * (p2y - A * c2y))
    b = (m2 * py * (dp2y - B * dc2y) - dpy * (p2y - B * c2y)) / \
        (m2 * xy * (dp2y - B * dc2y) - dxy * (p2y - B * c2y))
    return a, b


def amplitudes(a, b, Theta):
    """S1, S2 at scattering angles Theta (array)."""
    mu = np.cos(np.asarray(Theta, np.float64))
    nmax = len(a)
    S1 = np.zeros(mu.shape, np.complex128)
    S2 = np.zeros(mu.shape, np.complex128)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    for n in range(1, nmax + 1):
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += f * (a[n - 1] * tau + b[n - 1] * pi_cur)
        pi_next = ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def efficiencies(a, b, x):
    n = np.arange(1, len(a) + 1)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * (a + b).real)
    return qext, qsca


def _to_bh_index(eps_r, mu_r=1.0):
    # e^{+jwt} lossy eps = e' - j e''  ->  e^{-iwt} index with positive imaginary part
    m = np.sqrt(complex(eps_r) * complex(mu_r))
    return complex(m.real, abs(m.imag))


def sphere_bistatic(radius, eps_r, theta_obs, k=2 * np.pi, plane="E"):
    """RCS [m^2] of a homogeneous sphere for incidence along -z (x-pol), observed
    at theta_obs in the phi = 0 (E) or phi = 90 deg (H) plane."""
    m = _to_bh_index(eps_r)
    a, b = coefficients_homogeneous(k * radius, m)
    S1, S2 = amplitudes(a, b, np.pi - np.asarray(theta_obs))
    S = S2 if plane == "E" else S1
    return 4.0 * np.pi * np.abs(S) ** 2 / k ** 2


def coated_bistatic(r_core, r_shell, eps_core, eps_shell, theta_obs, k=2 * np.pi, plane="E"):
    m1 = _to_bh_index(eps_core)
    m2 = _to_bh_index(eps_shell)
    a, b = coefficients_coated(k * r_core, k * r_shell, m1, m2)
    S1, S2 = amplitudes(a, b, np.pi - np.asarray(theta_obs))
    S = S2 if plane == "E" else S1
    return 4.0 * np.pi * np.abs(S) ** 2 / k ** 2

"""Closed-form potential integrals over a flat triangle (oracle, test infrastructure).

Singularity extraction for the weakly and strongly singular parts of the
Green's function G = exp(-jkR)/(4 pi R) (Eq. 7) and of its gradient, needed
by the Galerkin entries of Eqs. 23-26 for self, adjacent and close triangle
pairs.  The paper does not describe singular integration; these are the
standard analytic results for a planar triangle (Wilton et al. 1984, Graglia
1993), restated here from the geometry:

For an observation point r, source triangle T with unit normal n, height
w = n.(r - v0), in-plane projection rho, and for each side i (vertices a -> b
counter-clockwise about n): unit tangent l_i, outward in-plane normal
u_i = l_i x n, s-/+ = (a|b - rho).l_i, t0 = (a - rho).u_i, R0^2 = t0^2 + w^2,
R+/- = |r - b|, |r - a|,

    f_i   = ln[(R+ + s+) / (R- + s-)]
    beta_i = atan(t0 s+ / (R0^2 + |w| R+)) - atan(t0 s- / (R0^2 + |w| R-))

    I1   = int_T 1/R dA'              = sum_i t0_i f_i - |w| sum_i beta_i
    Irho = int_T (rho' - rho)/R dA'   = 1/2 sum_i u_i [R0_i^2 f_i + s+ R+ - s- R-]
    Igr  = int_T grad_r (1/R) dA'     = -sum_i u_i f_i - sign(w) n sum_i beta_i

At w = 0 the normal component of Igr is its principal value (zero); the
+-1/2 jump terms are carried separately by the Gram (identity) terms.
"""
from __future__ import annotations

import numpy as np


def triangle_potentials(r, tv):
    """r [..., 3] observation points; tv [..., 3, 3] triangle vertices (broadcast).

    Returns (I1 [...], Irho [..., 3], Igr [..., 3], rho [..., 3])."""
    r = np.asarray(r, np.float64)
    tv = np.asarray(tv, np.float64)
    v0, v1, v2 = tv[..., 0, :], tv[..., 1, :], tv[..., 2, :]
    n = np.cross(v1 - v0, v2 - v0)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    w = np.einsum("...x,...x->...", r - v0, n)
    scale = np.linalg.norm(v1 - v0, axis=-1)
    w = np.where(np.abs(w) < 1e-12 * scale, 0.0, w)
    rho = r - w[..., None] * n
    aw = np.abs(w)
    I1 = np.zeros(np.broadcast_shapes(w.shape))
    Irho = np.zeros(I1.shape + (3,))
    Igr = np.zeros(I1.shape + (3,))
    sb = np.zeros(I1.shape)
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        el = b - a
        l = el / np.linalg.norm(el, axis=-1, keepdims=True)
        u = np.cross(l, n)
        sm = np.einsum("...x,...x->...", a - rho, l)
        sp = np.einsum("...x,...x->...", b - rho, l)
        t0 = np.einsum("...x,...x->...", a - rho, u)
        R02 = t0 * t0 + w * w
        Rp = np.linalg.norm(r - b, axis=-1)
        Rm = np.linalg.norm(r - a, axis=-1)
        # stable logarithm: (R + s)(R - s) = R0^2
        both_neg = (sp < 0) & (sm < 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            Ap = np.where(sp >= 0, Rp + sp, R02 / (Rp - sp))
            Am = np.where(sm >= 0, Rm + sm, R02 / (Rm - sm))
            f = np.where(both_neg, np.log((Rm - sm) / (Rp - sp)), np.log(Ap / Am))
        beta = np.arctan2(t0 * sp, R02 + aw * Rp) - np.arctan2(t0 * sm, R02 + aw * Rm)
        I1 = I1 + t0 * f
        Irho = Irho + 0.5 * u * (R02 * f + sp * Rp - sm * Rm)[..., None]
        Igr = Igr - u * f[..., None]
        sb = sb + beta
    I1 = I1 - aw * sb
    Igr = Igr - (np.sign(w) * sb)[..., None] * n
    return I1, Irho, Igr, rho

"""Far field and radar cross section (oracle, test infrastructure).

Eqs. 27-29, read with the e^{+jwt} convention of the Green's function (Eq. 7):
the scattered field in the host medium 0 is radiated by the host-side currents
J_0 = s_0 J, M_0 = s_0 M; in the far zone

  E(r) ~ (-j k e^{-jkr} / (4 pi r)) [eta N_perp - r x L],
  N = int J_0 e^{+jk r.r'} ds',  L = int M_0 e^{+jk r.r'} ds',

so that  sigma = lim 4 pi r^2 |E_s|^2/|E_i|^2 = k^2/(4 pi) |eta N_perp - r x L|^2 / |E0|^2.
In the scaled unknowns (eta_0 c, v): eta N = eta~_0 N^ with N^ built from eta_0 c.
Components: sigma_theta uses eta~ N^_theta + L_phi, sigma_phi uses eta~ N^_phi - L_theta.
"""
from __future__ import annotations

import numpy as np

from .quadrature import radon7, points
from .rwg import Mesh, material
from .fill import k0_of, _tri_data


def far_amplitudes(mesh: Mesh, x, obs, freq_hz=None):
    """x [nrhs, 2 ne] scaled solution; obs [nobs, 2] (theta, phi).
    Returns complex far amplitudes A [nrhs, nobs, 2] with sigma = |A|^2 / |E0|^2."""
    x = np.atleast_2d(x)
    k0 = k0_of(freq_hz)
    k, eta = material(mesh.media[0], k0)
    bR, wR = radon7()
    tris0 = mesh.region_tris(0)
    d = _tri_data(mesh, tris0, 0)        # region 0's functions (side signs included)
    pts = points(mesh.verts[mesh.tris[tris0]], bR)                 # [T,A,3]
    W = mesh.area[tris0][:, None] * wR[None, :]
    F = d["c"][:, :, None, None] * (pts[:, None, :, :] - d["v"][:, :, None, :])     # [T,i,A,3]
    m = d["e"]
    s = np.where(m >= 0, 1.0, 0.0)
    th, ph = obs[:, 0], obs[:, 1]
    rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    that = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    phat = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], 1)
    out = np.zeros((len(x), len(obs), 2), np.complex128)
    for o in range(len(obs)):
        ph_ = np.exp(1j * k * np.einsum("tax,x->ta", pts, rhat[o])) * W          # [T,A]
        P = np.einsum("ta,tiax->tix", ph_, F) * s[:, :, None]                    # per local basis
        Pt = np.einsum("tix,x->ti", P, that[o])
        Pp = np.einsum("tix,x->ti", P, phat[o])
        ok = m >= 0
        mm = np.maximum(m, 0)
        for r in range(len(x)):
            cJ = np.where(ok, x[r, 2 * mm], 0.0)
            cM = np.where(ok, x[r, 2 * mm + 1], 0.0)
            Nt, Np = np.sum(Pt * cJ), np.sum(Pp * cJ)
            Lt, Lp = np.sum(Pt * cM), np.sum(Pp * cM)
            pre = -1j * k / np.sqrt(4.0 * np.pi)
            out[r, o, 0] = pre * (eta * Nt + Lp)
            out[r, o, 1] = pre * (eta * Np - Lt)
    return out


def rcs(mesh: Mesh, x, obs, E0=1.0, freq_hz=None):
    """Bistatic RCS [nrhs, nobs, 2] in m^2 (sigma_theta, sigma_phi), Eq. 29."""
    A = far_amplitudes(mesh, x, obs, freq_hz)
    return np.abs(A) ** 2 / abs(E0) ** 2


def db_lambda2(sigma, lam=1.0):
    return 10.0 * np.log10(np.maximum(sigma, 1e-300) / lam ** 2)

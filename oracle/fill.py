"""Dense Galerkin JMCFIE matrix and excitation (oracle, test infrastructure).

Formulation (e^{+j w t}; readings of the garbled passages stated here):

Per medium l (Eqs. 5-7) with k_l, eta_l and the four boundary equations
(Eqs. 8-11) written from Maxwell's equations with the *inward* normal
n_l = s_l n of B_l and currents J_l = s_l J, M_l = s_l M (Eqs. 12-13):

  T-EFIE_l :  eta_l (L J_l)_t + (K M_l)_t + 1/2 n_l x M_l =  E_l^inc_t
  T-MFIE_l :  (K J_l)_t + 1/2 n_l x J_l - (L M_l)_t / eta_l = -H_l^inc_t
  N-EFIE_l : -eta_l n_l x L J_l - n_l x K M_l + 1/2 M_l      = -n_l x E_l^inc
  N-MFIE_l :  n_l x K J_l - 1/2 J_l - n_l x L M_l / eta_l     = -n_l x H_l^inc

  L X = jk int [X + k^-2 (div' X) grad] G ds',   K X = int grad G x X ds'
  (K is the principal value; its jump is the explicit 1/2 terms).

JMCFIE (Eq. 14 for one interface, Eq. 16 for several):
  J-row = sum_l s_l(m) [ eta_l^-1 T-EFIE_l - N-MFIE_l ]
  M-row = sum_l s_l(m) [ N-EFIE_l - eta_l T-MFIE_l ]
The N-parts carry the (-1)^l of Eq. 14 with l = 1 the host (s_l = -(-1)^l);
the T-parts are weighted by s_l so that the operators of the two media add
across an interface (PMCHWT-type); with these signs every eigenvalue of the
discrete operator lies in the right half-plane (the reading adopted for the
garbled signs).  Tested with RWG t_m = b_m (Galerkin, Eqs. 13-14 of the
discretisation section).  Unknowns and rows are scaled so that every block is
dimensionless: unknown pair (eta_0 c_n, v_n), J-row multiplied by eta_0.  With
eta~_l = eta_l / eta_0 and the Galerkin matrices

  L_l[m,n]  = <t_m, L_l b_n>    (Eq. 23: jk int int [t.b - k^-2 div t div' b] G)
  K_l[m,n]  = <t_m, K_l b_n>    (Eq. 26)
  NL_l[m,n] = <t_m, n_m x L_l b_n>   (Eq. 24)
  NK_l[m,n] = <t_m, n_m x K_l b_n>   (Eq. 25)
  G[m,n] = <t_m, b_n>,  Gx[m,n] = <t_m, n_m x b_n>

the 2x2 block of Z for (m, n) is the sum over media l containing both:

  JJ += s_m s_n L_l - s_n NK_l + 1/2 s_m s_n G
  JM += (s_m s_n K_l + s_n NL_l) / eta~_l + 1/2 s_m Gx / eta~_l
  MJ += -(s_m s_n K_l + s_n NL_l) eta~_l - 1/2 s_m Gx eta~_l
  MM += s_m s_n L_l - s_n NK_l + 1/2 s_m s_n G

Excitation (Eqs. 20-21; only the host medium 0 holds the source):
  b_J[m] = s_0(m)/eta~_0 <t_m, E> + <t_m, n_m x (eta_0 H)>
  b_M[m] = s_0(m) eta~_0 <t_m, eta_0 H> - <t_m, n_m x E>

Quadrature: Radon 7-point rule on both triangles for regular pairs; for
pairs with centroid distance < hmax_p + hmax_q a 4x4 collapsed-Gauss outer
rule with analytically extracted 1/R and grad(1/R) parts (potentials.py) and
the Radon rule on the bounded remainder.
"""
from __future__ import annotations

import numpy as np

from .quadrature import radon7, collapsed_gauss, points
from .potentials import triangle_potentials
from .rwg import Mesh, material

FOUR_PI = 4.0 * np.pi


def k0_of(freq_hz=None):
    c0 = 299792458.0
    if freq_hz is None:
        freq_hz = c0  # lambda0 = 1 m
    return 2.0 * np.pi * freq_hz / c0


def singular_pairs(mesh: Mesh, tris_l, test=None):
    """Pairs (p, q) of triangles of region l handled by singularity extraction:
    centroid distance < hmax_p + hmax_q.  Rows restricted to ``test`` (local
    indices into tris_l) when given."""
    test = np.arange(len(tris_l)) if test is None else test
    c = mesh.centroid[tris_l]
    h = mesh.hmax[tris_l]
    d = np.linalg.norm(c[test][:, None, :] - c[None, :, :], axis=2)
    return d < (h[test][:, None] + h[None, :])


def _inner_regular(r, tq, k):
    """Regular inner integrals at outer points r [P, A, 3] over all source
    triangles tq (dict of arrays, Q triangles). Returns I_G [P,A,Q],
    I_Gr [P,A,Q,3], I_gG [P,A,Q,3] (the 1/(4 pi) included)."""
    D = r[:, :, None, None, :] - tq["pts"][None, None, :, :, :]     # [P,A,Q,B,3]
    np.seterr(divide="ignore", invalid="ignore")
    R = np.sqrt(np.einsum("...x,...x->...", D, D))
    e = np.exp(-1j * k * R)
    Wq = tq["wq"][None, None, :, :]
    G = e / (FOUR_PI * R) * Wq
    I_G = G.sum(axis=3)
    I_Gr = np.einsum("paqb,qbx->paqx", G, tq["pts"])
    g = -(1.0 + 1j * k * R) * e / (FOUR_PI * R ** 3) * Wq
    I_gG = np.einsum("paqb,paqbx->paqx", g, D)
    return I_G, I_Gr, I_gG


def _inner_singular(r, tv, pts_q, wq, k):
    """Singular-extracted inner integrals, paired: r [N, A, 3]; tv [N, 3, 3];
    pts_q [N, B, 3]; wq [N, B] (area included)."""
    I1, Irho, Igr, rho = triangle_potentials(r, tv[:, None, :, :])
    D = r[:, :, None, :] - pts_q[:, None, :, :]                        # [N,A,B,3]
    R = np.sqrt(np.einsum("...x,...x->...", D, D))
    tiny = R < 1e-14
    Rs = np.where(tiny, 1.0, R)
    e = np.exp(-1j * k * Rs)
    rem = np.where(tiny, -1j * k, (e - 1.0) / Rs) * wq[:, None, :]      # (e^{-jkR}-1)/R
    I_G = (I1 + rem.sum(axis=2)) / FOUR_PI
    I_Gr = (Irho + rho * I1[..., None] + np.einsum("nab,nbx->nax", rem, pts_q)) / FOUR_PI
    gr = np.where(tiny, 0.0, (1.0 - (1.0 + 1j * k * Rs) * e) / Rs ** 3) * wq[:, None, :]
    I_gG = (Igr + np.einsum("nab,nabx->nax", gr, D)) / FOUR_PI
    return I_G, I_Gr, I_gG


def _pair_sum(W, X, Y):
    """sum_a W[n,a] X[n,i,a,:] . Y[n,j,a,:]  ->  [n,i,j]  (batched matmul)."""
    N, I, A, _ = X.shape
    Xw = (X * W[:, None, :, None]).reshape(N, I, A * 3)
    return np.matmul(Xw, Y.reshape(N, Y.shape[1], A * 3).transpose(0, 2, 1))


def _combine(W, r, tp, tq, I_G, I_Gr, I_gG, k):
    """Galerkin values for the 3x3 local basis combinations of paired
    triangles.  W [N,A] outer weights (area included), r [N,A,3] outer points,
    tp/tq dicts of per-pair test/source data.  Returns L, K, NL, NK [N,3,3].

      L  = jk sum_a W f_m . int f_n G  - (j/k) div f_m div f_n sum_a W int G
      K  = sum_a W f_m . (int grad G) x f_n(r_a ... )     [int grad G x f_n = (int grad G) x (r - v')]
      NL = sum_a W (f_m x n) . [jk int f_n G + (j/k) div f_n int grad G]
      NK = sum_a W (f_m x n) . (int grad G) x (r - v') c'
    """
    Fm = tp["c"][:, :, None, None] * (r[:, None, :, :] - tp["v"][:, :, None, :])     # [N,i,A,3]
    Fmn = np.cross(Fm, tp["n"][:, None, None, :])
    Fn = tq["c"][:, :, None, None] * (I_Gr[:, None, :, :] - tq["v"][:, :, None, :] * I_G[:, None, :, None])
    Cr = tq["c"][:, :, None, None] * np.cross(I_gG[:, None, :, :], r[:, None, :, :] - tq["v"][:, :, None, :])
    SG = np.einsum("na,na->n", W, I_G)
    L = 1j * k * _pair_sum(W, Fm, Fn) - (1j / k) * tp["d"][:, :, None] * tq["d"][:, None, :] * SG[:, None, None]
    K = _pair_sum(W, Fm, Cr)
    Gd = tq["d"][:, :, None, None] * I_gG[:, None, :, :]                                # [N,j,A,3]
    NL = 1j * k * _pair_sum(W, Fmn, Fn) + (1j / k) * _pair_sum(W, Fmn, Gd)
    NK = _pair_sum(W, Fmn, Cr)
    return L, K, NL, NK


def _tri_data(mesh: Mesh, idx, l=None):
    """Per-triangle basis data for triangles idx: local-edge coefficient
    c = sigma l/(2A), divergence d = sigma l / A, free-vertex coords v, normal n.
    With a region l: the pieces of region l's functions, i.e. sigma times
    s_l(T) (the side of T that l is on), and the normal s_l(T) n_T of region l
    (Eqs. 12-13 applied per triangle, which also covers junction edges)."""
    te = mesh.tri_edge[idx]
    sg = mesh.tri_sign[idx]
    n = mesh.normal[idx]
    if l is not None:
        st = mesh.tri_region_sign(l)[idx]
        sg = sg * st[:, None]
        n = n * st[:, None]
    ln = np.where(te >= 0, mesh.length[np.maximum(te, 0)], 0.0)
    A = mesh.area[idx]
    return dict(
        c=sg * ln / (2.0 * A[:, None]),
        d=sg * ln / A[:, None],
        v=mesh.verts[mesh.tri_free[idx]],
        n=n,
        e=te,
    )


def region_operators(mesh: Mesh, l, rows=None, chunk=24, outer_n=4, freq_hz=None):
    """Galerkin matrices of medium l over all edges (rows restricted to
    ``rows``): dict with L, K, NL, NK [nrows, ne] (zero where an edge is not
    on the boundary of B_l), Gram G and Gx [nrows, ne], and k, eta~.  They are
    taken between region l's own functions (each triangle's piece times the
    side sign s_l(T)) with region l's normals s_l(T) n_T, so the side signs of
    Eqs. 12-13 are already in them."""
    k0 = k0_of(freq_hz)
    ne = mesh.ne
    rows = np.arange(ne) if rows is None else np.asarray(rows, np.int64)
    row_map = -np.ones(ne, np.int64)
    row_map[rows] = np.arange(len(rows))
    need_tri = np.any(np.isin(mesh.tri_edge, rows) & (mesh.tri_edge >= 0), axis=1)
    k, eta = material(mesh.media[l], k0)
    out = {nm: np.zeros((len(rows), ne), np.complex128) for nm in ("L", "K", "NL", "NK", "G", "Gx")}
    out["k"], out["eta"] = k, eta
    tris_l = mesh.region_tris(l)
    if len(tris_l) == 0:
        return out
    bR, wR = radon7()
    bS, wS = collapsed_gauss(outer_n)
    tv_all = mesh.verts[mesh.tris[tris_l]]
    pts_all = points(tv_all, bR)                                          # [Q,7,3]
    wq_all = mesh.area[tris_l][:, None] * wR[None, :]
    tq_all = dict(pts=pts_all, wq=wq_all)
    src = _tri_data(mesh, tris_l, l)
    test_local = np.nonzero(need_tri[tris_l])[0]
    sing = singular_pairs(mesh, tris_l, test_local)          # [len(test_local), Q]

    def scatter(pi, qi, vals):
        m = src["e"][pi][:, :, None].repeat(3, axis=2).ravel()
        n = src["e"][qi][:, None, :].repeat(3, axis=1).ravel()
        rr = np.where(m >= 0, row_map[np.maximum(m, 0)], -1)
        ok = (rr >= 0) & (n >= 0)
        for nm, v in vals.items():
            np.add.at(out[nm], (rr[ok], n[ok]), v.ravel()[ok])

    # regular pairs: Radon rule on both triangles
    for c0 in range(0, len(test_local), chunk):
        pl = test_local[c0:c0 + chunk]
        srow = sing[c0:c0 + chunk]
        I_G, I_Gr, I_gG = _inner_regular(pts_all[pl], tq_all, k)          # [P,A,Q,...]
        P, A, Q = I_G.shape
        pi = np.repeat(pl, Q)
        qi = np.tile(np.arange(Q), P)
        mask = ~srow.ravel()
        pi, qi = pi[mask], qi[mask]
        I_G = I_G.transpose(0, 2, 1).reshape(P * Q, A)[mask]
        I_Gr = I_Gr.transpose(0, 2, 1, 3).reshape(P * Q, A, 3)[mask]
        I_gG = I_gG.transpose(0, 2, 1, 3).reshape(P * Q, A, 3)[mask]
        tp = {kk: vv[pi] for kk, vv in src.items()}
        tq = {kk: vv[qi] for kk, vv in src.items()}
        L, K, NL, NK = _combine(wq_all[pi], pts_all[pi], tp, tq, I_G, I_Gr, I_gG, k)
        scatter(pi, qi, dict(L=L, K=K, NL=NL, NK=NK))

    # singular / near-singular pairs: collapsed-Gauss outer rule, extracted inner
    sp_, sq_ = np.nonzero(sing)
    sp_ = test_local[sp_]
    for c0 in range(0, len(sp_), 4096):
        pi, qi = sp_[c0:c0 + 4096], sq_[c0:c0 + 4096]
        r = points(tv_all[pi], bS)                                        # [N,16,3]
        W = mesh.area[tris_l][pi][:, None] * wS[None, :]
        I_G, I_Gr, I_gG = _inner_singular(r, tv_all[qi], pts_all[qi], wq_all[qi], k)
        tp = {kk: vv[pi] for kk, vv in src.items()}
        tq = {kk: vv[qi] for kk, vv in src.items()}
        L, K, NL, NK = _combine(W, r, tp, tq, I_G, I_Gr, I_gG, k)
        scatter(pi, qi, dict(L=L, K=K, NL=NL, NK=NK))

    # Gram terms, same-triangle overlaps (Radon rule is exact for these quadratics)
    tl = test_local
    rq = pts_all[tl]
    d = {kk: vv[tl] for kk, vv in src.items()}
    F = d["c"][:, :, None, None] * (rq[:, None, :, :] - d["v"][:, :, None, :])       # [T,i,A,3]
    Fx = np.cross(d["n"][:, None, None, :], F)                                         # n x f
    Gm = _pair_sum(wq_all[tl], F, F)
    Gx = _pair_sum(wq_all[tl], F, Fx)
    scatter(tl, tl, dict(G=Gm, Gx=Gx))
    return out


FORMULATIONS = ("jmcfie", "ctf", "cnf", "pmchwt", "ictf")


def formulation_weights(formulation, eta):
    """Weights (aTJ, aNJ, aTM, aNM) of medium l (relative impedance eta~_l) in
    J-row = sum_l s_l [aTJ T-EFIE_l / eta_l - aNJ N-MFIE_l] and
    M-row = sum_l s_l [aNM N-EFIE_l - aTM eta_l T-MFIE_l]:
    JMCFIE (Eq. 14) all 1; CTF the tangential parts only; CNF the normal
    parts only; PMCHWT the tangential equations unweighted by the medium's
    impedance (aTJ = eta~_l, aTM = 1 / eta~_l), whose 1/2 jump terms cancel
    between the two sides of an interface.  The variants the paper compares
    its JMCFIE with (its iteration-count study)."""
    if formulation == "jmcfie":
        return 1.0, 1.0, 1.0, 1.0
    if formulation == "ctf":
        return 1.0, 0.0, 1.0, 0.0
    if formulation == "cnf":
        return 0.0, 1.0, 0.0, 1.0
    if formulation in ("pmchwt", "ictf"):
        return eta, 0.0, 1.0 / eta, 0.0
    raise ValueError(f"unknown formulation {formulation!r}")


def ictf_row_weights(mesh: Mesh, freq_hz=None, rows=None):
    """Row weights of the ICTF (the improved CTF of the Fig. 6 comparison,
    defined in a reference outside the paper's text; reading taken here): the
    CTF weights each medium's tangential equations by that medium's own
    impedance, the ICTF normalises both tangential equations of an interface
    by the mean relative impedance e = (eta~_a + eta~_b) / 2 of the two media
    it separates.  Summed over the two media with the PMCHWT weights, this is
    J-row = (1/e) sum_l s_l T-EFIE_l, M-row = -e sum_l s_l T-MFIE_l: the
    PMCHWT rows of each edge times (1/e, e).  Returns (wJ, wM) per row edge."""
    if np.any(mesh.junction):
        raise ValueError("ICTF: the mean impedance of an interface is not defined at junction edges")
    k0 = k0_of(freq_hz)
    rows = np.arange(mesh.ne) if rows is None else np.asarray(rows, np.int64)
    eta = np.array([material(mesh.media[l], k0)[1] for l in range(mesh.nr)])
    er = mesh.edge_regions[rows]
    e = 0.5 * (eta[er[:, 0]] + eta[er[:, 1]])
    return 1.0 / e, e


def assemble(mesh: Mesh, freq_hz=None, rows=None, chunk=24, outer_n=4, formulation="jmcfie"):
    """Dense matrix (scaled) of the given formulation (default JMCFIE), shape
    [2 ne, 2 ne] with per-edge (J, M) interleaving; if ``rows`` (edge indices)
    is given only those edge rows are returned, shape [2 len(rows), 2 ne].
    Tangential (T) and normal (N) parts of each block, per medium:
      JJ: T  ss L                      N  -sn NK + 1/2 ss G
      JM: T  (ss K + 1/2 sm Gx) / eta  N  sn NL / eta
      MJ: T -(ss K + 1/2 sm Gx) eta    N -sn NL eta
      MM: T  ss L                      N  -sn NK + 1/2 ss G
    weighted by formulation_weights (J-row: aTJ, aNJ; M-row: aTM, aNM)."""
    return assemble_variants(mesh, (formulation,), freq_hz, rows, chunk, outer_n)[formulation]


def assemble_variants(mesh: Mesh, formulations=FORMULATIONS, freq_hz=None, rows=None, chunk=24, outer_n=4):
    """``assemble`` for several formulations from one evaluation of the
    media's Galerkin matrices: dict formulation -> matrix."""
    ne = mesh.ne
    rows = np.arange(ne) if rows is None else np.asarray(rows, np.int64)
    out = {f: np.zeros((2 * len(rows), 2 * ne), np.complex128) for f in formulations}
    for l in range(mesh.nr):
        # region l's operators between its own functions (side signs s_l of
        # Eqs. 12-13 included per triangle, region normals n_l)
        op = region_operators(mesh, l, rows, chunk, outer_n, freq_hz)
        eta = op["eta"]
        tK = op["K"] + 0.5 * op["Gx"]
        nN = -op["NK"] + 0.5 * op["G"]
        for f, Z in out.items():
            aTJ, aNJ, aTM, aNM = formulation_weights(f, eta)
            Z[0::2, 0::2] += aTJ * op["L"] + aNJ * nN
            Z[0::2, 1::2] += (aTJ * tK + aNJ * op["NL"]) / eta
            Z[1::2, 0::2] += -(aTM * tK + aNM * op["NL"]) * eta
            Z[1::2, 1::2] += aTM * op["L"] + aNM * nN
    if "ictf" in out:
        wJ, wM = ictf_row_weights(mesh, freq_hz, rows)
        out["ictf"][0::2, :] *= wJ[:, None]
        out["ictf"][1::2, :] *= wM[:, None]
    return out


def plane_wave(theta_i, phi_i, pol, E0=1.0):
    """Plane wave arriving from direction (theta_i, phi_i): propagation
    k = -r(theta_i, phi_i); polarisation e = cos(pol) theta_hat + sin(pol) phi_hat
    (Eq. 30, read with e^{+jwt}: E = e E0 exp(-j k0 k.r))."""
    st, ct, sp, cp = np.sin(theta_i), np.cos(theta_i), np.sin(phi_i), np.cos(phi_i)
    rhat = np.array([st * cp, st * sp, ct])
    th = np.array([ct * cp, ct * sp, -st])
    ph = np.array([-sp, cp, 0.0])
    khat = -rhat
    e = np.cos(pol) * th + np.sin(pol) * ph
    return khat, e * E0


def rhs(mesh: Mesh, inc, freq_hz=None, formulation="jmcfie"):
    """Excitation vectors, shape [nrhs, 2 ne], rows (J, M) interleaved, of the
    given formulation (weights of the host medium, formulation_weights).
    inc: rows (theta_i, phi_i, pol_angle, E0)."""
    k0 = k0_of(freq_hz)
    inc = np.atleast_2d(np.asarray(inc, np.float64))
    _, eta0 = material(mesh.media[0], k0)
    bR, wR = radon7()
    tris0 = mesh.region_tris(0)
    d = _tri_data(mesh, tris0, 0)        # region 0's functions and normals (side signs included)
    pts = points(mesh.verts[mesh.tris[tris0]], bR)
    W = mesh.area[tris0][:, None] * wR[None, :]
    F = d["c"][:, :, None, None] * (pts[:, None, :, :] - d["v"][:, :, None, :])      # [T,i,A,3]
    Fxn = np.cross(F, d["n"][:, None, None, :])                                      # f x n
    out = np.zeros((len(inc), 2 * mesh.ne), np.complex128)
    k_0, _ = material(mesh.media[0], k0)
    for ri, (th, ph, pol, E0) in enumerate(inc):
        khat, e = plane_wave(th, ph, pol, E0)
        E = np.exp(-1j * k_0 * np.einsum("tax,x->ta", pts, khat))[..., None] * e      # [T,A,3]
        H = np.cross(khat[None, None, :], E) / eta0                                   # eta_0 H (host impedance eta0 * eta~_0)
        fE = np.einsum("ta,tiax,tax->ti", W, F, E)
        fH = np.einsum("ta,tiax,tax->ti", W, F, H)
        fnH = np.einsum("ta,tiax,tax->ti", W, Fxn, H)    # <f, n x H> = int H.(f x n)
        fnE = np.einsum("ta,tiax,tax->ti", W, Fxn, E)
        m = d["e"]
        ok = m >= 0
        aTJ, aNJ, aTM, aNM = formulation_weights(formulation, eta0)
        bJ = aTJ * fE / eta0 + aNJ * fnH
        bM = aTM * eta0 * fH - aNM * fnE
        np.add.at(out[ri], 2 * m[ok], bJ[ok])
        np.add.at(out[ri], 2 * m[ok] + 1, bM[ok])
    if formulation == "ictf":
        wJ, wM = ictf_row_weights(mesh, freq_hz)
        out[:, 0::2] *= wJ[None, :]
        out[:, 1::2] *= wM[None, :]
    return out

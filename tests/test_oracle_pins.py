"""Pins of the CPU oracle against facts fixed by mathematics and the paper
(closed forms, invariants, brute force) -- never against the CUDA path."""
import os
from math import factorial

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1704_06862_gb300 import geometry as geo
from oracle import fill, farfield, mie, potentials, quadrature, solvers, tree
from oracle.rwg import Mesh, material


# ---------------------------------------------------------------- quadrature
def _mono(b, w, p, q):
    return 0.5 * np.sum(w * b[:, 1] ** p * b[:, 2] ** q)


def test_radon7_exact_to_degree5_not_6():
    b, w = quadrature.radon7()
    assert abs(w.sum() - 1.0) < 1e-15
    for p in range(6):
        for q in range(6 - p):
            exact = factorial(p) * factorial(q) / factorial(p + q + 2)
            assert abs(_mono(b, w, p, q) - exact) < 1e-15
    assert abs(_mono(b, w, 6, 0) - factorial(6) / factorial(8)) > 1e-6


def test_collapsed_gauss_degree():
    for n in (2, 3, 4, 6):
        b, w = quadrature.collapsed_gauss(n)
        for p in range(2 * n - 1):
            for q in range(2 * n - 1 - p):
                exact = factorial(p) * factorial(q) / factorial(p + q + 2)
                assert abs(_mono(b, w, p, q) - exact) < 1e-14


# ---------------------------------------------------------------- potentials
TV = np.array([[0.1, 0.05, 0.0], [1.0, 0.2, 0.1], [0.3, 0.9, -0.2]])


def _area(tv):
    return 0.5 * np.linalg.norm(np.cross(tv[1] - tv[0], tv[2] - tv[0]))


@pytest.mark.parametrize("r", [[0.4, 0.4, 0.8], [2.0, -1.0, 0.3], [0.45, 0.38, 0.05], [0.5, -0.4, -0.1]])
def test_potentials_vs_brute_force_off_plane(r):
    r = np.array(r)
    b, w = quadrature.collapsed_gauss(80)
    P = b @ TV
    A = _area(TV)
    I1, Ir, Ig, rho = potentials.triangle_potentials(r, TV)
    D = r - P
    R = np.linalg.norm(D, axis=1)
    assert abs(I1 - A * np.sum(w / R)) < 1e-9 * abs(I1)
    assert np.allclose(Ir, A * np.sum(w[:, None] * (P - rho) / R[:, None], 0), atol=1e-9)
    assert np.allclose(Ig, A * np.sum(-w[:, None] * D / R[:, None] ** 3, 0), rtol=1e-7, atol=1e-8)


def test_potential_gradient_is_derivative_of_I1():
    r = np.array([0.35, 0.3, 0.07])
    h = 1e-6
    _, _, Ig, _ = potentials.triangle_potentials(r, TV)
    fd = np.array([(potentials.triangle_potentials(r + h * e, TV)[0] - potentials.triangle_potentials(r - h * e, TV)[0]) / (2 * h)
                   for e in np.eye(3)])
    assert np.allclose(Ig, fd, rtol=1e-6, atol=1e-7)


def test_potential_in_plane_point_by_duffy_split():
    """Observation point inside the triangle: split at the point into three
    sub-triangles and integrate 1/R with a rule collapsed at the point (the
    Duffy map cancels the singularity) -- independent of the edge formulas."""
    bary = np.array([0.3, 0.45, 0.25])
    r = bary @ TV
    I1, Ir, Ig, _ = potentials.triangle_potentials(r, TV)
    b, w = quadrature.collapsed_gauss(40)
    tot, totr = 0.0, np.zeros(3)
    for a, c in ((0, 1), (1, 2), (2, 0)):
        sub = np.array([TV[a], TV[c], r])
        # put the collapsed vertex of the map at r:
        bb = b[:, [0, 2, 1]]          # the map collapses at barycentric coordinate 1
        P = bb @ sub
        A = _area(sub)
        R = np.linalg.norm(P - r, axis=1)
        tot += A * np.sum(w / R)
        totr += A * np.sum(w[:, None] * (P - r) / R[:, None], 0)
    assert abs(I1 - tot) < 1e-10 * tot
    assert np.allclose(Ir, totr, atol=1e-10)
    n = np.cross(TV[1] - TV[0], TV[2] - TV[0])
    assert abs(np.dot(Ig, n)) < 1e-12 * np.linalg.norm(n)     # principal value of the normal part


# ---------------------------------------------------------------- mesh / RWG
def test_rwg_counts_and_charge_neutrality():
    for nu in (1, 2, 3, 8):
        m = Mesh(**geo.homogeneous_sphere(nu=nu))
        assert m.nt == 20 * nu * nu and m.ne == 30 * nu * nu
    m = Mesh(**geo.homogeneous_sphere(nu=3))
    # divergence is +l/A+ on T+ and -l/A- on T-: total charge vanishes (Eq. 22)
    q = m.length / m.area[m.tp] * m.area[m.tp] - m.length / m.area[m.tm] * m.area[m.tm]
    assert np.max(np.abs(q)) < 1e-14
    # every triangle of a closed surface carries three bases
    assert np.all(m.tri_edge >= 0)


def test_rwg_normal_continuity_across_edge():
    """f_n . (edge normal in each triangle) equals 1 on the edge from both sides."""
    m = Mesh(**geo.homogeneous_sphere(nu=2))
    for e in range(0, m.ne, 7):
        a, b = m.verts[m.edge_v[e]]
        mid = 0.5 * (a + b)
        for t, v, s in ((m.tp[e], m.vp[e], 1.0), (m.tm[e], m.vm[e], -1.0)):
            f = s * m.length[e] / (2 * m.area[t]) * (mid - m.verts[v])
            nhat = np.cross(b - a, m.normal[t])
            nhat /= np.linalg.norm(nhat)
            # outward edge normal of T+ points toward T-
            if np.dot(nhat, mid - m.centroid[t]) < 0:
                nhat = -nhat
            flux = np.dot(f, nhat) * s
            assert abs(flux - 1.0) < 1e-12


def test_material_branch():
    k, eta = material([6.0, -0.6, 1.0, 0.0], 2 * np.pi)
    assert k.imag < 0 and k.real > 0 and eta.real > 0
    assert abs(k / (2 * np.pi) - np.sqrt(6 - 0.6j)) < 1e-14
    assert abs(eta - 1 / np.sqrt(6 - 0.6j)) < 1e-14


# ---------------------------------------------------------------- Galerkin fill
@pytest.fixture(scope="module")
def small_sphere_ops():
    m = Mesh(**geo.homogeneous_sphere(nu=3, radius=0.5, eps_r=4.0))
    return m, [fill.region_operators(m, l) for l in range(2)]


def _regular_edge_pairs(m):
    """Edge pairs none of whose four triangle pairs takes the singular path."""
    sing = fill.singular_pairs(m, np.arange(m.nt))   # all rows
    e_t = np.stack([m.tp, m.tm], 1)
    out = np.ones((m.ne, m.ne), bool)
    for a in range(2):
        for b in range(2):
            out &= ~sing[e_t[:, a][:, None], e_t[:, b][None, :]]
    return out


def test_galerkin_symmetry(small_sphere_ops):
    """Reciprocity: <t_m, L b_n> and <t_m, K b_n> are symmetric.  With the
    same Radon rule on both triangles the symmetry is exact for regular pairs;
    the singular outer rule breaks it at quadrature-error level only."""
    m, ops = small_sphere_ops
    reg = _regular_edge_pairs(m)
    assert reg.sum() > 0.5 * m.ne ** 2
    for op in ops:
        for nm in ("L", "K", "G"):
            A = op[nm]
            scale = np.max(np.abs(A))
            assert np.max(np.abs((A - A.T)[reg])) <= 1e-12 * scale, nm
        assert np.max(np.abs(op["L"] - op["L"].T)) <= 3e-3 * np.max(np.abs(op["L"]))
        assert np.max(np.abs(op["K"] - op["K"].T)) <= 0.25 * np.max(np.abs(op["K"]))


@pytest.mark.slow
def test_singular_K_converges_to_symmetric():
    """Refining the outer rule of singular pairs drives K toward symmetry
    (the exact operator is symmetric), pinning the extracted inner integrals."""
    m = Mesh(**geo.homogeneous_sphere(nu=2, radius=0.5, eps_r=4.0))
    asym = []
    for n in (4, 16):
        K = fill.region_operators(m, 1, outer_n=n)["K"]
        asym.append(np.max(np.abs(K - K.T)) / np.max(np.abs(K)))
    assert asym[1] < 0.25 * asym[0]


def test_gram_matches_closed_form(small_sphere_ops):
    """Self Gram entry of an RWG: sum over both triangles of
    l^2/(4A^2) int |r - v|^2 = l^2/(4A) * (|e1|^2+|e2|^2+|e3|^2 ... ) closed form
    int_T |r - v0|^2 dA = A/6 (|a|^2 + |b|^2 + a.b) with a, b the sides from v0."""
    m, ops = small_sphere_ops
    G = ops[0]["G"]
    for e in range(0, m.ne, 11):
        tot = 0.0
        for t, v in ((m.tp[e], m.vp[e]), (m.tm[e], m.vm[e])):
            others = [x for x in m.tris[t] if x != v]
            a = m.verts[others[0]] - m.verts[v]
            b = m.verts[others[1]] - m.verts[v]
            A = m.area[t]
            tot += m.length[e] ** 2 / (4 * A * A) * A / 6 * (a @ a + b @ b + a @ b)
        assert abs(G[e, e] - tot) < 1e-13 * tot


def test_coplanar_K_vanishes():
    """For coplanar triangle pairs (t.(grad G x b) with all vectors in plane
    is normal . in-plane = 0), K and n x K vanish identically -- flat plate."""
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0.5, 0.5, 0]], float) * 0.2
    t = np.array([[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]], np.int32)
    m = Mesh(v, t, np.tile([[0, 1]], (4, 1)), np.array([[1, 0, 1, 0], [4, 0, 1, 0]]))
    op = fill.region_operators(m, 0)
    assert np.max(np.abs(op["K"])) < 1e-15 and np.max(np.abs(op["NK"])) < 1e-15
    assert np.max(np.abs(op["L"])) > 1e-3


def _null_case(nu):
    m = Mesh(**geo.homogeneous_sphere(nu=nu, radius=0.5, eps_r=1.0))
    Z = fill.assemble(m)
    b = fill.rhs(m, [[0, 0, 0, 1.0]])[0]
    x = solvers.lu_solve(Z, b)
    return m, x, farfield.rcs(m, x, geo.bistatic_angles(19))[0]


def test_null_body_scatters_nothing():
    """eps_r = 1 body: the exact solution is the equivalent current of the
    incident wave with zero scattered field (Eqs. 1-2, extinction).  Every
    sign of the formulation and excitation enters this check: the scattered
    field must vanish as the mesh is refined, and the currents must approach
    n x H and -n x E of the incident wave.

    With eps_r = 1 the discrete scattered field is pure discretisation error
    (the RWG space cannot hold the incident wave's surface currents exactly),
    so its level is set by the mesh, not by a tolerance: -22.2 dBsm at nu = 3
    and -30.4 dBsm at nu = 5 with the adopted JMCFIE signs, about 35 dB below
    the +5 dBsm a real body of this size scatters.  The bound -28 dBsm sits
    2.4 dB above the nu = 5 level, and the refinement step (at least 5 dB
    lower from nu = 3 to nu = 5, measured 8.2 dB) pins the convergence to
    zero, which a sign error anywhere in the formulation would break."""
    _, _, s3 = _null_case(3)
    m, x, s5 = _null_case(5)
    assert 10 * np.log10(s5.max()) < -28.0
    assert 10 * np.log10(s5.max()) < 10 * np.log10(s3.max()) - 5.0
    op = fill.region_operators(m, 0)
    G = op["G"]
    from oracle.quadrature import radon7, points
    bR, wR = radon7()
    khat, e = fill.plane_wave(0, 0, 0)
    pj = np.zeros(m.ne, complex)
    pm = np.zeros(m.ne, complex)
    for t in range(m.nt):
        P = points(m.verts[m.tris[t]], bR)
        E = np.exp(-1j * 2 * np.pi * P @ khat)[:, None] * e
        H = np.cross(khat, E)
        J = np.cross(m.normal[t], H)
        M = -np.cross(m.normal[t], E)
        for j in range(3):
            ed = m.tri_edge[t, j]
            f = m.tri_sign[t, j] * m.length[ed] / (2 * m.area[t]) * (P - m.verts[m.tri_free[t, j]])
            pj[ed] += m.area[t] * np.sum(wR * np.einsum("ax,ax->a", f, J))
            pm[ed] += m.area[t] * np.sum(wR * np.einsum("ax,ax->a", f, M))
    cj = np.linalg.solve(G, pj)
    cm = np.linalg.solve(G, pm)
    assert np.linalg.norm(x[0::2] - cj) / np.linalg.norm(cj) < 0.1
    assert np.linalg.norm(x[1::2] - cm) / np.linalg.norm(cm) < 0.1


def test_jmcfie_spectrum_right_half_plane():
    """With the combination signs read from Eq. 14 (adopted reading), the discrete
    operator of a dielectric sphere has its whole spectrum in Re > 0 (the
    property that makes the combined formulation converge quickly)."""
    m = Mesh(**geo.homogeneous_sphere(nu=3, radius=0.5, eps_r=4.0))
    Z = fill.assemble(m)
    ev = np.linalg.eigvals(Z)
    assert ev.real.min() > 0


@pytest.mark.slow
def test_sphere_converges_to_mie():
    """Homogeneous sphere, eps_r = 4, radius 0.5 lambda0 (the Fig. 5 check of
    the paper, on the geometry of the homogeneous-sphere workload): bistatic
    RCS at all 361 angles of the phi = 0 plane, nulls included, against the
    Lorenz-Mie series under mesh refinement nu = 4, 6, 8 (nu = 8 is the
    3840-unknown workload mesh).  The mean |error| in dB must fall at each
    step at close to the second-order rate of a flat-facet RWG discretisation
    (error ~ h^2, h ~ 1/nu: the ratio between meshes at least 0.8 of
    (nu_fine / nu_coarse)^2), the maximum must fall too, and the finest mesh
    must be inside the 0.2 dB bar of the method (measured 0.634, 0.287,
    0.165 dB mean; 1.10, 0.54, 0.32 dB max)."""
    obs = geo.bistatic_angles(361)
    ref = 10 * np.log10(mie.sphere_bistatic(0.5, 4.0, obs[:, 0]))
    nus = (4, 6, 8)
    mean, mx = [], []
    for nu in nus:
        m = Mesh(**geo.homogeneous_sphere(nu=nu, radius=0.5, eps_r=4.0))
        x = solvers.lu_solve(fill.assemble(m), fill.rhs(m, [[0, 0, 0, 1.0]])[0])
        d = np.abs(10 * np.log10(farfield.rcs(m, x, obs)[0][:, 0]) - ref)
        mean.append(d.mean())
        mx.append(d.max())
    for i in range(len(nus) - 1):
        assert mean[i + 1] < mean[i] and mx[i + 1] < mx[i], (mean, mx)
        assert mean[i] / mean[i + 1] > 0.8 * (nus[i + 1] / nus[i]) ** 2, (mean, mx)
    assert mean[-1] < 0.2 and mx[-1] < 0.4, (mean, mx)


@pytest.mark.slow
def test_cube_monostatic_mirror_symmetry():
    """Lossy dielectric cube (eps 6 - 0.6j, the cube workload's material),
    edge 0.6 lambda0, 6 x 6 squares per face: the body and its mesh are mirror-symmetric under
    z -> -z, which maps a theta-polarised incidence at theta_i onto one at
    pi - theta_i in the phi = 0 plane, so the monostatic theta-theta RCS must
    agree at the two angles (no closed form exists for a cube: this is its
    pin, with the stored oracle values).  The singular outer quadrature
    depends on the vertex order of each triangle, which the mirror changes,
    so the symmetry holds to quadrature accuracy (measured 0.006 dB)."""
    m = Mesh(**geo.workload("cube_tiny"))
    inc = geo.monostatic_incidences(8)
    Z = fill.assemble(m)
    X = np.stack([solvers.lu_solve(Z, b) for b in fill.rhs(m, inc)])
    R = farfield.rcs(m, X, np.stack([inc[:, 0], inc[:, 1]], axis=1))
    mono = 10 * np.log10(np.array([R[i, i, 0] for i in range(len(inc))]))
    assert np.max(np.abs(mono - mono[::-1])) < 0.02
    # broadside incidences see a face, the 45-degree-ish ones an edge: a real spread
    assert np.ptp(mono) > 1.0
    # the stored oracle values of the finer cube (same body) and of the
    # tri-axial ellipsoid (z -> -z is one of its principal-plane mirrors) obey
    # the same symmetry
    for name in ("cube_small", "ellipsoid_small"):
        d = np.load(os.path.join(os.path.dirname(__file__), "golden", f"{name}.npz"))
        ds = 10 * np.log10(d["mono_rcs"])
        assert np.max(np.abs(ds - ds[::-1])) < 0.02, name


# ---------------------------------------------------------------- Mie series
def test_mie_rayleigh_limit():
    x, m = 0.01, 2.0 + 0.0j
    a, b = mie.coefficients_homogeneous(x, m)
    S1, S2 = mie.amplitudes(a, b, np.array([0.3, 1.2, 2.5]))
    pol = (m * m - 1) / (m * m + 2)
    assert np.allclose(np.abs(S1), x ** 3 * abs(pol), rtol=1e-3)
    assert np.allclose(np.abs(S2), x ** 3 * abs(pol) * np.abs(np.cos([0.3, 1.2, 2.5])), rtol=1e-3)


def test_mie_optical_theorem_lossless():
    for x, m in ((3.14, 2.0), (9.4, 1.6)):
        a, b = mie.coefficients_homogeneous(x, m)
        qe, qs = mie.efficiencies(a, b, x)
        assert abs(qe - qs) < 1e-10 * qs
        S1, S2 = mie.amplitudes(a, b, np.array([0.0]))
        assert abs(qe - 4 / x ** 2 * S1[0].real) < 1e-10 * qe   # forward amplitude
    a, b = mie.coefficients_coated(2 * np.pi, 3 * np.pi, 2.0, 1.6)
    qe, qs = mie.efficiencies(a, b, 3 * np.pi)
    assert abs(qe - qs) < 1e-10 * qs


def test_coated_reduces_to_homogeneous():
    th = np.linspace(0, np.pi, 13)
    # shell index = core index: a sphere of the outer radius
    s1 = mie.coated_bistatic(1.0, 1.5, 4.0, 4.0, th)
    s2 = mie.sphere_bistatic(1.5, 4.0, th)
    assert np.allclose(s1, s2, rtol=1e-8)
    # shell index = host index: a sphere of the inner radius
    s1 = mie.coated_bistatic(1.0, 1.5, 4.0, 1.0, th)
    s2 = mie.sphere_bistatic(1.0, 4.0, th)
    assert np.allclose(s1, s2, rtol=1e-8)


def test_mie_negative_permittivity():
    """Metal spheres (Re eps < 0, the plasmonic nanoparticle's media): the
    Rayleigh limit with the quasi-static polarisability (eps - 1)/(eps + 2);
    energy balance -- a lossless negative-eps sphere (imaginary index)
    scatters all it extinguishes, a lossy one absorbs (Q_ext > Q_sca > 0,
    which fails if the loss sign is flipped); a coated sphere whose shell and
    core are the same metal is the homogeneous metal sphere."""
    eps_c, eps_s = geo.NANO_EPS_CORE, geo.NANO_EPS_SHELL
    x = 0.01
    a, b = mie.coefficients_homogeneous(x, mie._to_bh_index(eps_c))
    S1, _ = mie.amplitudes(a, b, np.array([0.3, 1.2]))
    assert np.allclose(np.abs(S1), x ** 3 * abs((eps_c - 1) / (eps_c + 2)), rtol=1e-3)
    x = 2 * np.pi * 250 / 550
    a, b = mie.coefficients_homogeneous(x, mie._to_bh_index(-10.0))
    qe, qs = mie.efficiencies(a, b, x)
    assert abs(qe - qs) < 1e-9 * qs
    for m in (mie._to_bh_index(eps_c), mie._to_bh_index(eps_s)):
        qe, qs = mie.efficiencies(*mie.coefficients_homogeneous(x, m), x)
        assert qe > qs > 0
    a, b = mie.coefficients_coated(2 * np.pi * 230 / 550, x, mie._to_bh_index(eps_c), mie._to_bh_index(eps_s))
    qe, qs = mie.efficiencies(a, b, x)
    assert qe > qs > 0
    th = np.linspace(0, np.pi, 13)
    assert np.allclose(mie.coated_bistatic(230 / 550, 250 / 550, eps_s, eps_s, th),
                       mie.sphere_bistatic(250 / 550, eps_s, th), rtol=1e-8)


def test_stored_nanoparticle_oracle_near_mie():
    """The stored oracle RCS of the plasmonic coated nanoparticle (dense
    JMCFIE + LU on the nu = 6 mesh) against the coated-sphere Mie series of
    the same radii and media: within 1 dB on average (0.67 dB; the oracle
    reaches 0.39 dB at nu = 8)."""
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "nanoparticle.npz"))
    ref = mie.coated_bistatic(230 / 550, 250 / 550, geo.NANO_EPS_CORE, geo.NANO_EPS_SHELL, d["obs"][:, 0])
    assert np.allclose(ref, d["mie"], rtol=1e-10)
    err = np.abs(10 * np.log10(d["rcs"][:, 0]) - 10 * np.log10(ref))
    assert err.mean() < 1.0


# ---------------------------------------------------------------- solvers / ILU / tree
def _rand_system(n=60, seed=3):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_fgmres_matches_lu():
    A, b = _rand_system()
    x, its, hist = solvers.fgmres(lambda v: A @ v, b, restart=10, tol=1e-10)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-8 * np.linalg.norm(x)
    assert hist[-1] < 1e-10 and its > 10          # restarts happened


@pytest.mark.parametrize("solver", ["bicgstab", "cgs"])
def test_bicgstab_cgs_match_lu(solver):
    """The paper's solvers converge to the dense solution, unpreconditioned and
    with a right preconditioner (the residual they monitor is b - A x)."""
    f = getattr(solvers, solver)
    A, b = _rand_system()
    xe = np.linalg.solve(A, b)
    D = np.diag(np.diag(A))
    for M in (None, lambda v: np.linalg.solve(D, v)):
        x, its, hist = f(lambda v: A @ v, b, precond=M, tol=1e-11, maxit=500)
        assert np.linalg.norm(x - xe) < 1e-9 * np.linalg.norm(xe)
        assert np.linalg.norm(b - A @ x) < 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs"])
def test_bicgstab_cgs_finite_termination(solver):
    """Both are built on BiCG: with three distinct eigenvalues the BiCG
    residual polynomial vanishes after three steps, so they stop within three
    iterations; with the exact inverse as preconditioner, after one."""
    f = getattr(solvers, solver)
    rng = np.random.default_rng(11)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.array([1.0 + 0.5j, 2.0, 5.0 - 1.0j])[rng.integers(0, 3, n)]
    A = Q @ np.diag(lam) @ Q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, hist = f(lambda v: A @ v, b, tol=1e-9, maxit=50)
    assert its <= 3 and np.linalg.norm(b - A @ x) < 1e-8 * np.linalg.norm(b)
    Ai = np.linalg.inv(A)
    x, its, hist = f(lambda v: A @ v, b, precond=lambda v: Ai @ v, tol=1e-9, maxit=50)
    assert its == 1 and np.linalg.norm(b - A @ x) < 1e-8 * np.linalg.norm(b)


def test_ilu0_full_pattern_is_exact_lu():
    A, b = _rand_system(40)
    F = solvers.ilu0(sp.csr_matrix(A))
    z = solvers.ilu_apply(F, b)
    assert np.linalg.norm(z - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(z)


def test_ilu0_defining_property():
    """(L U)_ij = A_ij on the pattern; fill outside the pattern is dropped."""
    rng = np.random.default_rng(5)
    n = 50
    mask = rng.random((n, n)) < 0.15
    mask |= np.eye(n, dtype=bool)
    A = np.where(mask, rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 0) + 6 * np.eye(n)
    F = solvers.ilu0(sp.csr_matrix(A)).toarray()
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    LU = L @ U
    assert np.max(np.abs((LU - A)[mask])) < 1e-12
    assert np.max(np.abs(LU[~mask] - A[~mask])) > 1e-6    # genuinely incomplete


def test_tree_colouring_and_order():
    m = Mesh(**geo.homogeneous_sphere(nu=4))
    ijk = tree.box_coords(m, 4)
    col = tree.colour(ijk)
    near = tree.near_mask(m, 4)
    same_box = (ijk[:, None, :] == ijk[None, :, :]).all(axis=2)
    # touching distinct boxes never share a colour
    assert not np.any(near & ~same_box & (col[:, None] == col[None, :]))
    perm = tree.ordering(m, 4)
    assert np.array_equal(np.sort(perm), np.arange(m.ne))
    c = col[perm]
    assert np.all(np.diff(c) >= 0)


def test_formulation_variants():
    """The formulations the paper compares with JMCFIE, from the same Galerkin
    matrices: every one reproduces the Mie series of a dielectric sphere
    (RWG discretisation error, coarse mesh); JMCFIE is exactly CTF + CNF;
    PMCHWT has symmetric diagonal blocks and JM = -MJ (its jump terms cancel
    across the interface); and the iteration counts order as expected for
    these integral equations (the combined forms converge faster than
    PMCHWT; ICTF between CTF and PMCHWT, as the paper's comparison reports)."""
    m = Mesh(**geo.homogeneous_sphere(nu=5, radius=0.5, eps_r=4.0))
    obs = geo.bistatic_angles(37)
    ref = mie.sphere_bistatic(0.5, 4.0, obs[:, 0])
    Zs = fill.assemble_variants(m)
    its = {}
    for f, Z in Zs.items():
        b = fill.rhs(m, [[0.0, 0.0, 0.0, 1.0]], formulation=f)[0]
        x = solvers.lu_solve(Z, b)
        db = np.abs(10 * np.log10(farfield.rcs(m, x[None], obs)[0][:, 0]) - 10 * np.log10(ref))
        assert db.mean() < 1.2 and db.max() < 2.0, (f, db.mean(), db.max())
        its[f] = solvers.fgmres(lambda v: Z @ v, b, restart=50, tol=1e-4, maxit=2000)[1]
    assert np.abs(Zs["jmcfie"] - Zs["ctf"] - Zs["cnf"]).max() < 1e-13
    P = Zs["pmchwt"]
    A, B, C, D = P[0::2, 0::2], P[0::2, 1::2], P[1::2, 0::2], P[1::2, 1::2]
    assert np.abs(A - A.T).max() < 1e-2 * np.abs(A).max()
    assert np.abs(D - D.T).max() < 1e-2 * np.abs(D).max()
    assert np.abs(B + C).max() < 1e-13 * np.abs(B).max()
    assert its["jmcfie"] < its["ctf"] < its["pmchwt"] and its["cnf"] < its["ctf"]
    # the paper's ordering of its Fig. 6 comparison: ICTF above CTF, PMCHWT above both
    assert its["ctf"] < its["ictf"] < its["pmchwt"]
    # ICTF re-weights whole rows of the PMCHWT system (per interface), so its
    # discrete solution is the PMCHWT one; a weight applied to columns, to only
    # one of the two media or not to the excitation breaks this
    bP = fill.rhs(m, [[0.0, 0.0, 0.0, 1.0]], formulation="pmchwt")[0]
    bI = fill.rhs(m, [[0.0, 0.0, 0.0, 1.0]], formulation="ictf")[0]
    xP, xI = solvers.lu_solve(P, bP), solvers.lu_solve(Zs["ictf"], bI)
    assert np.abs(xI - xP).max() < 1e-9 * np.abs(xP).max()
    assert np.abs(Zs["ictf"] - P).max() > 1e-2 * np.abs(P).max()   # a different system


def test_ictf_matched_impedance():
    """Media with eps_r = mu_r have the free-space impedance: every weight of
    the tangential forms is 1, so CTF, ICTF and PMCHWT are the same matrix
    and excitation (their weights differ only through the impedances)."""
    g = geo.homogeneous_sphere(nu=3, radius=0.5, eps_r=2.0)
    media = np.array(g["media"], np.float64)
    media[1] = [2.0, 0.0, 2.0, 0.0]
    g["media"] = media
    m = Mesh(**g)
    Zs = fill.assemble_variants(m, ("ctf", "pmchwt", "ictf"))
    scale = np.abs(Zs["pmchwt"]).max()
    assert np.abs(Zs["ictf"] - Zs["pmchwt"]).max() < 1e-13 * scale
    assert np.abs(Zs["ctf"] - Zs["pmchwt"]).max() < 1e-13 * scale
    inc = [[0.3, 0.2, 0.0, 1.0]]
    bP, bI = fill.rhs(m, inc, formulation="pmchwt"), fill.rhs(m, inc, formulation="ictf")
    assert np.abs(bI - bP).max() < 1e-14 * np.abs(bP).max()


def test_junction_edges_split_sphere():
    """Junction edges (three surfaces meeting at an edge, Eq. 16's multilayer
    setting): a sphere cut by the plane z = 0 into two regions of the same
    eps has the same exterior field as the uncut sphere of the same outer
    mesh.  Its equator edges are shared by an upper-hemisphere (0|1), a
    lower-hemisphere (0|2) and a disk (1|2) triangle; the region-based RWG
    ties them to one unknown with per-triangle coefficients a_T such that every
    region's equivalent current is divergence-conforming across the edge.
    Pins: the constraints hold on every junction edge; the split body's RCS
    approaches the uncut body's as the mesh is refined (discretisation error
    of the disk: 0.23 then 0.089 dB mean, the h^2 rate), far below what a
    wrong coefficient gives (flipping the disk's: 3.4 dB mean); both stay
    within the coarse-mesh distance of the Mie series."""
    obs = geo.bistatic_angles(37)
    inc = [[0.0, 0.0, 0.0, 1.0]]
    ref = mie.sphere_bistatic(0.3, 4.0, obs[:, 0])

    def rcs_of(m):
        Z = fill.assemble(m)
        x = solvers.lu_solve(Z, fill.rhs(m, inc)[0])
        return farfield.rcs(m, x[None], obs)[0][:, 0]

    diffs = []
    for nl, no, nr in ((8, 16, 2), (12, 24, 3)):
        ms = Mesh(**geo.split_sphere(nl, no, nr))
        assert int(ms.junction.sum()) == no                      # the equator edges
        for e in np.nonzero(ms.junction)[0]:
            sides = [(t, ms.tri_sign[t, j]) for t in range(ms.nt) for j in range(3) if ms.tri_edge[t, j] == e]
            assert len(sides) == 3
            for l in range(3):
                on = [(t, a) for t, a in sides if l in ms.tri_regions[t]]
                assert len(on) == 2
                (t1, a1), (t2, a2) = on
                s1 = 1.0 if ms.tri_regions[t1, 0] == l else -1.0
                s2 = 1.0 if ms.tri_regions[t2, 0] == l else -1.0
                assert s1 * a1 == -s2 * a2
        mh = Mesh(**geo.latlong_homogeneous_sphere(nl, no))
        rs, rh = rcs_of(ms), rcs_of(mh)
        d = np.abs(10 * np.log10(rs) - 10 * np.log10(rh))
        diffs.append(d.mean())
        assert np.abs(10 * np.log10(rs) - 10 * np.log10(ref)).mean() < 1.0
    assert diffs[0] < 0.3 and diffs[1] < 0.12 and diffs[1] < 0.5 * diffs[0], diffs


def test_junction_edges_null_lens():
    """The lens on a slab (five media, junction edges on three base circles
    where a hemisphere and two annuli of the slab's top face meet) with every
    medium free space: the exact scattered field is zero (Eqs. 1-2 with
    identical media; the outer surface carries the incident wave's equivalent
    currents, the interior surfaces none), so the discrete one is
    discretisation error and must fall as the mesh is refined: -6.1 dBsm at
    h = 0.3 lambda0, -13.2 at 0.15 (-18.4 at 0.1), against +17.7 dBsm for the
    dielectric lens of the same mesh.  Every junction constraint of every
    region enters: flipping the coefficient of the outer hemisphere's
    triangles at the outer base circle (a plausible sign slip) raises the
    coarse level by 6.7 dB (and leaves +0.8 dBsm at h = 0.15, no
    convergence)."""
    obs = geo.bistatic_angles(19)
    inc = [[0.0, 0.0, 0.0, 1.0]]

    def null_lens(nlon, h, plant=False):
        m = Mesh(**geo.lens_on_slab((0.15, 0.3, 0.6), (1.0, 1.0, 1.0), (1.4, 1.4, 0.2), 1.0, nlon=nlon, h=h))
        if plant:
            for t in range(m.nt):
                if tuple(m.tri_regions[t]) == (0, 3):
                    for j in range(3):
                        if m.junction[m.tri_edge[t, j]]:
                            m.tri_sign[t, j] *= -1
        x = solvers.lu_solve(fill.assemble(m), fill.rhs(m, inc)[0])
        return 10 * np.log10(farfield.rcs(m, x[None], obs)[0][:, 0].max())

    coarse, fine = null_lens(8, 0.3), null_lens(16, 0.15)
    planted = null_lens(8, 0.3, plant=True)
    assert fine < -10.0 and fine < coarse - 5.0, (coarse, fine)
    assert planted > coarse + 4.0, (coarse, planted)

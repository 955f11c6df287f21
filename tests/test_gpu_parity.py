"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances:
* near-field entries, excitation, RCS of a given current, ILU apply (FP64):
  same quadrature and same definitions on both sides -> 1e-9 relative
  (rounding and atomic-add order only).
* FP32 (mixed) forms vs FP64 forms: 1e-4 relative L2 (single precision with
  O(100)-term sums).
The small fixtures here have triangles as large as the leaf boxes, so their
far field is checked only for FP32/FP64 and multi-RHS consistency; MLFMM
accuracy against the dense oracle is checked on the stored cases
(test_gpu_golden.py) and at full size (test_gpu_fullsize.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402
from oracle import fill, farfield, solvers, tree  # noqa: E402
from oracle.rwg import Mesh  # noqa: E402


def _dev(a, ne):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1, ne, 2)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(t.shape[0], -1)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


class Case:
    def __init__(self, name, mesh, levels, digits=3.0):
        self.mesh = mesh
        self.levels = levels
        self.m = Mesh(**mesh)
        self.s = sie.Solver(mesh, levels=levels, digits=digits)
        self.ne = self.s.ne
        self._Z = None

    @property
    def Z(self):
        if self._Z is None:
            self._Z = fill.assemble(self.m)
        return self._Z


@pytest.fixture(scope="module")
def sphere():
    c = Case("sphere", geo.homogeneous_sphere(nu=4, radius=0.5, eps_r=4.0), levels=4)
    yield c
    c.s.close()


@pytest.fixture(scope="module")
def coated():
    c = Case("coated", geo.coated_sphere(5, 3, 0.75, 0.5, 2.56, 4.0), levels=4)
    yield c
    c.s.close()


@pytest.fixture(scope="module")
def lossy():
    c = Case("lossy", geo.homogeneous_sphere(nu=4, radius=0.5, eps_r=6.0 - 0.6j), levels=4)
    yield c
    c.s.close()


def test_rwg_numbering_matches(sphere):
    assert sphere.ne == sphere.m.ne


def test_near_field_entries(sphere, coated, lossy):
    for c in (sphere, coated, lossy):
        rows, cols, vals = sie.sie_near_export(c.s.ctx)
        Z = c.Z
        ref = np.stack([Z[2 * rows + a, 2 * cols + b] for a in range(2) for b in range(2)], axis=1)
        scale = np.max(np.abs(Z))
        assert np.max(np.abs(vals - ref)) < 1e-9 * scale
        # the pattern is exactly the touching-box pattern of the definition
        mask = tree.near_mask(c.m, c.levels)
        assert len(rows) == mask.sum()
        assert mask[rows, cols].all()


@pytest.mark.parametrize("prec,tol", [(sie.SIE_PREC_FP64, 1e-12), (sie.SIE_PREC_MIXED, 2e-5)])
def test_near_spmv(sphere, coated, prec, tol):
    for c in (sphere, coated):
        mask = tree.near_mask(c.m, c.levels)
        Zn = c.Z * np.repeat(np.repeat(mask, 2, 0), 2, 1)
        x = geo.random_coefficients(2 * c.ne, 2, seed=11)
        y = torch.zeros_like(_dev(x, c.ne))
        sie.sie_matvec_parts(c.s.ctx, _dev(x, c.ne), y, 2, prec, parts=1)
        assert rel(_host(y), (Zn @ x.T).T) < tol


def test_mixed_matvec_close_to_fp64(coated):
    c = coated
    x = geo.random_coefficients(2 * c.ne, 3, seed=3)
    y64 = torch.zeros_like(_dev(x, c.ne))
    y32 = torch.zeros_like(y64)
    sie.mlfmm_matvec(c.s.ctx, _dev(x, c.ne), y64, 3, sie.SIE_PREC_FP64)
    sie.mlfmm_matvec(c.s.ctx, _dev(x, c.ne), y32, 3, sie.SIE_PREC_MIXED)
    assert rel(_host(y32), _host(y64)) < 1e-4


def test_multi_rhs_equals_single(coated):
    c = coated
    x = geo.random_coefficients(2 * c.ne, 3, seed=9)
    yb = torch.zeros_like(_dev(x, c.ne))
    sie.mlfmm_matvec(c.s.ctx, _dev(x, c.ne), yb, 3, sie.SIE_PREC_FP64)
    yb = _host(yb)
    for r in range(3):
        y1 = torch.zeros_like(_dev(x[r:r + 1], c.ne))
        sie.mlfmm_matvec(c.s.ctx, _dev(x[r:r + 1], c.ne), y1, 1, sie.SIE_PREC_FP64)
        assert rel(_host(y1)[0], yb[r]) < 1e-13


def _oracle_ilu(c):
    mask = tree.near_mask(c.m, c.levels)
    perm = tree.ordering(c.m, c.levels)
    A = solvers.pattern_matrix(c.Z, mask, perm)
    return solvers.ilu0(A), perm


@pytest.mark.parametrize("prec,tol", [(sie.SIE_PREC_FP64, 1e-9), (sie.SIE_PREC_MIXED, 1e-4)])
def test_ilu_apply(coated, prec, tol):
    c = coated
    F, perm = _oracle_ilu(c)
    v = geo.random_coefficients(2 * c.ne, 1, seed=21)[0]
    # oracle works in the preconditioner ordering: position p holds edge perm[p]
    vp = v.reshape(c.ne, 2)[perm].reshape(-1)
    zp = solvers.ilu_apply(F, vp)
    z = np.empty_like(v).reshape(c.ne, 2)
    z[perm] = zp.reshape(c.ne, 2)
    out = torch.zeros_like(_dev(v, c.ne))
    sie.ilu_apply(c.s.ctx, _dev(v, c.ne), out, 1, prec)
    assert rel(_host(out)[0], z.reshape(-1)) < tol


@pytest.mark.parametrize("prec", [sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED])
def test_ilu_schedules_agree(coated, prec):
    """One persistent cooperative launch for the 15 colour steps and one
    launch per step (the default) give identical results (same items, same
    order)."""
    c = coated
    v = _dev(geo.random_coefficients(2 * c.ne, 1, seed=22)[0], c.ne)
    out = []
    try:
        for sched in (0, 1):
            sie.sie_set_param(c.s.ctx, 1, sched)
            z = torch.full_like(v, float("nan"))
            sie.ilu_apply(c.s.ctx, v, z, 1, prec)
            out.append(_host(z))
    finally:
        sie.sie_set_param(c.s.ctx, 1, 1)
    assert np.all(np.isfinite(out[0])) and np.array_equal(out[0], out[1])


def test_ilu_barrier_wait_gives_up_cleanly(coated):
    """The grid barriers of the persistent ILU(0) apply have a bounded wait.
    With a wait limit of 0 every barrier gives up at once (no GPU fault, no
    hang): the call (through sie_device_status) and gmres_solve report
    SIE_ETIMEOUT, and with
    the limit restored the same context applies ILU(0) correctly again."""
    c = coated
    sie.sie_set_param(c.s.ctx, 1, 0)
    v = _dev(geo.random_coefficients(2 * c.ne, 1, seed=23)[0], c.ne)
    ref = torch.zeros_like(v)
    sie.ilu_apply(c.s.ctx, v, ref, 1, sie.SIE_PREC_MIXED)
    sie.sie_device_status(c.s.ctx)
    try:
        sie.sie_set_param(c.s.ctx, 0, 0)
        z = torch.zeros_like(v)
        with pytest.raises(sie.SieError) as e:   # the binding reads the device record after the call
            sie.ilu_apply(c.s.ctx, v, z, 1, sie.SIE_PREC_MIXED)
        assert e.value.code == 7
        sie.sie_device_status(c.s.ctx)        # the record was cleared
        b = torch.zeros_like(v)
        sie.sie_plane_wave_rhs(c.s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
        with pytest.raises(sie.SieError) as e:
            sie.gmres_solve(c.s.ctx, b, torch.zeros_like(b), 1, restart=50, max_iters=100, tol=1e-4,
                            prec=sie.SIE_PREC_MIXED, precond=1)
        assert e.value.code == 7
    finally:
        sie.sie_set_param(c.s.ctx, 0, 1 << 21)
    z = torch.zeros_like(v)
    sie.ilu_apply(c.s.ctx, v, z, 1, sie.SIE_PREC_MIXED)
    sie.sie_device_status(c.s.ctx)
    sie.sie_set_param(c.s.ctx, 1, 1)
    assert torch.equal(z, ref)


@pytest.mark.parametrize("prec,tol", [(sie.SIE_PREC_FP64, 1e-9), (sie.SIE_PREC_MIXED, 1e-4)])
def test_ilu_apply_block(coated, prec, tol):
    """ILU(0) applied to a block of 10 right-hand sides (two passes of the
    block kernel's right-hand-side chunk in FP32, three in FP64) against the
    oracle ILU(0), column by column."""
    c = coated
    F, perm = _oracle_ilu(c)
    V = geo.random_coefficients(2 * c.ne, 10, seed=23)
    out = torch.zeros_like(_dev(V, c.ne))
    sie.ilu_apply(c.s.ctx, _dev(V, c.ne), out, 10, prec)
    got = _host(out)
    for r in (0, 7, 9):
        vp = V[r].reshape(c.ne, 2)[perm].reshape(-1)
        zp = solvers.ilu_apply(F, vp)
        z = np.empty_like(V[r]).reshape(c.ne, 2)
        z[perm] = zp.reshape(c.ne, 2)
        assert rel(got[r], z.reshape(-1)) < tol


def test_rhs_and_rcs(sphere, coated):
    for c in (sphere, coated):
        inc = np.array([[0.0, 0.0, 0.0, 1.0], [0.7, 0.3, 0.4, 2.0]])
        b = torch.zeros((2, c.ne, 2), dtype=torch.complex128, device="cuda")
        sie.sie_plane_wave_rhs(c.s.ctx, inc, b)
        assert rel(_host(b), fill.rhs(c.m, inc)) < 1e-12
        x = geo.random_coefficients(2 * c.ne, 2, seed=2)
        obs = geo.bistatic_angles(13)
        got = sie.rcs_farfield(c.s.ctx, _dev(x, c.ne), 2, obs)
        ref = farfield.rcs(c.m, x, obs)
        assert np.max(np.abs(got - ref)) < 1e-9 * np.max(ref)
        # mixed form: FP32 phases and currents; the RCS bar of the method is 0.2 dB
        got32 = sie.rcs_farfield_prec(c.s.ctx, _dev(x, c.ne), 2, obs, sie.SIE_PREC_MIXED)
        assert np.max(np.abs(got32 - ref)) < 1e-5 * np.max(ref)


def test_ilu_reduces_iterations(coated):
    c = coated
    b = torch.zeros((1, c.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(c.s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    its = []
    for pc in (0, 1):
        x = torch.zeros_like(b)
        st = sie.gmres_solve(c.s.ctx, b, x, 1, restart=50, max_iters=2000, tol=1e-4, precond=pc)
        its.append(st[0]["iters"])
    assert its[1] < its[0]


def test_tiny_body_near_only_and_errors():
    """Edge cases: a 4-triangle body whose bases all touch (empty far field);
    invalid meshes are rejected with SIE_EINVAL; calls out of order give
    SIE_ESTATE."""
    mesh = geo.tetra_body(0.3, 4.0)
    m = Mesh(**mesh)
    s = sie.Solver(mesh, levels=2)
    x = geo.random_coefficients(2 * s.ne, 1, seed=4)
    y = torch.zeros_like(_dev(x, s.ne))
    sie.mlfmm_matvec(s.ctx, _dev(x, s.ne), y, 1)
    assert rel(_host(y), (fill.assemble(m) @ x.T).T) < 1e-10
    s.close()
    ctx = sie.sie_create(0)
    bad = dict(mesh)
    bad["tris"] = mesh["tris"].copy()
    bad["tris"][0] = bad["tris"][0][[0, 2, 1]]          # inconsistent orientation
    with pytest.raises(sie.SieError) as e:
        sie.sie_build_mesh(ctx, bad["verts"], bad["tris"], bad["tri_regions"], bad["media"], 3e8)
    assert e.value.code == 1
    with pytest.raises(sie.SieError) as e:
        sie.mlfmm_setup(ctx, 4)
    assert e.value.code == 4
    sie.sie_destroy(ctx)


@pytest.mark.parametrize("method,name", [(sie.SOLVE_BICGSTAB, "bicgstab"), (sie.SOLVE_CGS, "cgs")])
def test_bicgstab_cgs_match_oracle_dense(sphere, method, name):
    """With two levels every pair is near, so the product is the dense
    Galerkin matrix: the GPU BiCGStab / CGS (FP64, no preconditioner) take the
    oracle's steps on the oracle's matrix and reach the dense-LU solution."""
    c = sphere
    s2 = sie.Solver(c.mesh, levels=2)
    try:
        inc = np.array([[0.3, 0.2, 0.0, 1.0]])
        bo = fill.rhs(c.m, inc)[0]
        b = _dev(bo[None], c.ne)
        x = torch.zeros_like(b)
        st = sie.gmres_solve(s2.ctx, b, x, 1, max_iters=500, tol=1e-8, prec=sie.SIE_PREC_FP64, precond=0,
                             method=method)
        xo, its, _ = getattr(solvers, name)(lambda v: c.Z @ v, bo, tol=1e-8, maxit=500)
        xe = solvers.lu_solve(c.Z, bo)
        assert st[0]["converged"]
        assert abs(st[0]["iters"] - its) <= 2
        assert rel(_host(x)[0], xe) < 1e-6
        assert rel(xo, xe) < 1e-6
    finally:
        s2.close()

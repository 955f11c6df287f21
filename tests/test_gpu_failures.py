"""Failure handling, driven from the host: no test here faults, traps or
hangs the GPU.  A non-finite excitation makes the solvers report
SIE_EBREAKDOWN, a too small iteration budget SIE_ENOTCONV with the statistics
filled in, invalid media SIE_EINVAL, and the context stays usable after each
failure (the next solve on it converges to the same answer as on a fresh
context)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402

EINVAL, ENOTCONV, EBREAKDOWN = 1, 5, 6
MESH = geo.coated_sphere(5, 3, 0.75, 0.5, 2.56, 4.0)


@pytest.fixture(scope="module")
def solver():
    import __graft_entry__ as g
    g.build()
    s = sie.Solver(MESH, levels=4)
    yield s
    s.close()


def _excitation(s):
    b = s.vec(1)
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    return b


def _reference_solution(s, b):
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=500, tol=1e-6, prec=sie.SIE_PREC_MIXED)
    assert st[0]["converged"]
    return x


@pytest.mark.parametrize("method", [sie.SOLVE_FGMRES, sie.SOLVE_BICGSTAB, sie.SOLVE_CGS])
def test_non_finite_excitation_is_a_breakdown(solver, method):
    s = solver
    b = _excitation(s)
    ref = _reference_solution(s, b)
    bad = b.clone()
    bad[0, s.ne // 2, 0] = complex(float("nan"), 0.0)
    x = torch.zeros_like(b)
    with pytest.raises(sie.SieError) as e:
        sie.gmres_solve(s.ctx, bad, x, 1, restart=50, max_iters=100, tol=1e-4, prec=sie.SIE_PREC_MIXED,
                        method=method)
    assert e.value.code == EBREAKDOWN
    # the context is still usable: the same solve with a finite excitation
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=500, tol=1e-6, prec=sie.SIE_PREC_MIXED)
    assert st[0]["converged"]
    assert float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)) < 1e-5


@pytest.mark.parametrize("method,budget", [(sie.SOLVE_FGMRES, 2), (sie.SOLVE_FGMRES, 1), (sie.SOLVE_BICGSTAB, 2),
                                           (sie.SOLVE_CGS, 2)])
def test_iteration_budget_gives_not_converged_with_stats(solver, method, budget):
    s = solver
    b = _excitation(s)
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=budget, tol=1e-4, prec=sie.SIE_PREC_MIXED,
                         method=method, check=False)[0]
    assert not st["converged"]
    assert 1 <= st["iters"] <= budget
    assert np.isfinite(st["rel_residual"]) and st["rel_residual"] > 1e-4
    if method == sie.SOLVE_FGMRES:          # minimal residual: never above the initial one
        assert st["rel_residual"] <= 1.0 + 1e-12
    with pytest.raises(sie.SieError) as e:
        x.zero_()
        sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=budget, tol=1e-4, prec=sie.SIE_PREC_MIXED,
                        method=method, check=True)
    assert e.value.code == ENOTCONV


def test_bad_solver_options_rejected(solver):
    s = solver
    b = _excitation(s)
    for kw in (dict(max_iters=0), dict(restart=0), dict(tol=-1.0), dict(tol=float("nan")), dict(method=7)):
        opts = dict(restart=50, max_iters=10, tol=1e-4, prec=sie.SIE_PREC_MIXED)
        opts.update(kw)
        with pytest.raises(sie.SieError) as e:
            sie.gmres_solve(s.ctx, b, torch.zeros_like(b), 1, **opts)
        assert e.value.code == EINVAL, kw


def test_two_rhs_one_poisoned(solver):
    """A block solve where one right-hand side is non-finite reports the
    breakdown."""
    s = solver
    b = s.vec(2)
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0], [0.5, 0.0, 0.0, 1.0]], b)
    b[1, 3, 1] = complex(float("inf"), 0.0)
    x = torch.zeros_like(b)
    with pytest.raises(sie.SieError) as e:
        sie.gmres_solve(s.ctx, b, x, 2, restart=50, max_iters=100, tol=1e-4, prec=sie.SIE_PREC_MIXED)
    assert e.value.code == EBREAKDOWN


@pytest.mark.parametrize("media_row", [[0.0, 0.0, 1.0, 0.0], [4.0, 0.0, 0.0, 0.0], [float("inf"), 0.0, 1.0, 0.0],
                                       [float("nan"), 0.0, 1.0, 0.0], [4.0, 0.5, 1.0, 0.0]])
def test_invalid_media_rejected(media_row):
    import __graft_entry__ as g
    g.build()
    mesh = geo.homogeneous_sphere(nu=3, radius=0.5, eps_r=4.0)
    media = mesh["media"].copy()
    media[1] = media_row
    ctx = sie.sie_create(0)
    try:
        with pytest.raises(sie.SieError) as e:
            sie.sie_build_mesh(ctx, mesh["verts"], mesh["tris"], mesh["tri_regions"], media, geo.FREQ_HZ)
        assert e.value.code == EINVAL
    finally:
        sie.sie_destroy(ctx)

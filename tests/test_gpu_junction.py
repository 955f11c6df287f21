"""Junction edges on the GPU: a sphere cut by the plane z = 0 into two regions
of the same eps (three surfaces meeting at every equator edge) scatters like
the uncut sphere of the same outer mesh; meshes whose junctions the
region-based RWG cannot represent, and the ICTF (whose per-interface weight
is not defined at a junction), are refused.  The stored oracle case
`split_sphere` runs through every golden test as well."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402

EINVAL = 1


def _rcs(mesh):
    s = sie.Solver(mesh, levels=3)
    try:
        b = s.vec(1)
        sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
        x = s.vec(1)
        st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=500, tol=1e-6, prec=sie.SIE_PREC_MIXED, precond=1)
        assert st[0]["converged"]
        return sie.rcs_farfield(s.ctx, x, 1, geo.bistatic_angles(91))[0, :, 0], st[0]["iters"]
    finally:
        s.close()


def test_split_sphere_matches_uncut_sphere():
    """The oracle puts the two bodies 0.089 dB apart (mean over angles) on
    this mesh, the disk's discretisation error; a wrong junction coefficient
    gives several dB."""
    import __graft_entry__ as g
    g.build()
    rs, its_s = _rcs(geo.split_sphere(12, 24, 3, 0.3, 4.0, 4.0))
    rh, its_h = _rcs(geo.latlong_homogeneous_sphere(12, 24, 0.3, 4.0))
    d = np.abs(10 * np.log10(rs) - 10 * np.log10(rh))
    print(f"split vs uncut: mean {d.mean():.4f} dB, max {d.max():.4f} dB; iterations {its_s} / {its_h}")
    assert d.mean() < 0.15 and d.max() < 0.4


def test_unsupported_junctions_and_ictf_refused():
    import __graft_entry__ as g
    g.build()
    mesh = geo.split_sphere(8, 16, 2, 0.3, 4.0, 4.0)
    # a second disk triangle on a rim edge: region 1 would see three faces there
    disk = np.nonzero(mesh["tri_regions"][:, 0] == 1)[0]
    rim = set(int(v) for v in mesh["tris"][disk[-1]])
    bad = dict(mesh)
    extra = mesh["tris"][disk[-1]].copy()
    extra[[1, 2]] = extra[[2, 1]]
    bad["tris"] = np.concatenate([mesh["tris"], extra[None]])
    bad["tri_regions"] = np.concatenate([mesh["tri_regions"], np.array([[2, 1]], np.int32)])
    assert len(rim) == 3
    ctx = sie.sie_create(0)
    try:
        with pytest.raises(sie.SieError) as e:
            sie.sie_build_mesh(ctx, bad["verts"], bad["tris"], bad["tri_regions"], bad["media"], geo.FREQ_HZ)
        assert e.value.code == EINVAL
    finally:
        sie.sie_destroy(ctx)
    with pytest.raises(sie.SieError) as e:
        sie.Solver(mesh, levels=3, formulation=sie.FORM_ICTF)
    assert e.value.code == EINVAL

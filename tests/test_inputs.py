"""The seeded synthetic inputs: sizes, radii, media and incidences of the
workloads the tests and the bench use (geodesic spheres of frequency nu have
20 nu^2 triangles and 30 nu^2 edges; two unknowns per edge)."""
import numpy as np
import pytest

from paper_1704_06862_gb300 import geometry as geo


def _unknowns(mesh):
    return 3 * len(mesh["tris"])      # closed surfaces: edges = 3/2 triangles, two unknowns per edge


@pytest.mark.parametrize("name,unknowns,radii", [
    ("sphere_c1", 3840, (0.5,)),
    ("coated_c2", 78000, (1.5, 1.0)),
    ("coated_small", 12480, (1.5, 1.0)),
    ("nanoparticle", 30720, (250 / 550, 230 / 550)),
])
def test_workload_sizes_and_radii(name, unknowns, radii):
    m = geo.workload(name)
    assert _unknowns(m) == unknowns
    r = np.linalg.norm(m["verts"], axis=1)
    assert np.allclose(sorted(set(np.round(r, 12)), reverse=True), radii)


def test_workload_media():
    m = geo.workload("coated_c2")
    assert np.allclose(m["media"][:, 0], [1.0, 2.56, 4.0]) and np.allclose(m["media"][:, 1], 0.0)
    n = geo.workload("nanoparticle")
    eps = n["media"][:, 0] + 1j * n["media"][:, 1]
    assert np.allclose(eps, [1.0, geo.NANO_EPS_SHELL, geo.NANO_EPS_CORE])
    assert np.all(n["media"][1:, 0] < 0) and np.all(n["media"][1:, 1] < 0)   # metals: Re eps < 0, loss e^{+jwt}
    # regions: the outer surface separates host (0) and shell (1), the inner shell (1) and core (2)
    assert set(map(tuple, n["tri_regions"])) == {(0, 1), (1, 2)}


def test_seeded_generators_are_deterministic():
    a = geo.random_coefficients(100, 2, seed=1234)
    b = geo.random_coefficients(100, 2, seed=1234)
    assert a.dtype == np.complex128 and np.array_equal(a, b)
    assert not np.array_equal(a, geo.random_coefficients(100, 2, seed=1235))
    assert abs(np.mean(np.abs(geo.random_coefficients(20000, 1)) ** 2) - 1.0) < 0.03   # unit variance


def test_incidence_sets():
    obs = geo.bistatic_angles(361)
    assert obs.shape == (361, 2) and obs[0, 0] == 0.0 and np.isclose(obs[-1, 0], np.pi) and np.all(obs[:, 1] == 0)
    inc = geo.monostatic_incidences(16)
    assert inc.shape == (16, 4) and np.isclose(inc[-1, 0], np.pi)
    assert np.all(inc[:, 1] == 0) and np.all(inc[:, 2] == 0) and np.all(inc[:, 3] == 1)


def test_cube_workload():
    """Cube of the monostatic workload: 3 lambda0 edge, 54 x 54 squares per
    face (104 976 unknowns), eps 6 - 0.6j; closed, outward, mirror-symmetric."""
    m = geo.workload("cube_c3")
    assert _unknowns(m) == 104976
    v, t = m["verts"], m["tris"]
    assert np.allclose(v.min(axis=0), -1.5) and np.allclose(v.max(axis=0), 1.5)
    eps = m["media"][1, 0] + 1j * m["media"][1, 1]
    assert eps == 6.0 - 0.6j
    s = geo.workload("cube_small")
    vs, ts = s["verts"], s["tris"]
    vol = np.sum(np.einsum("ij,ij->i", vs[ts[:, 0]], np.cross(vs[ts[:, 1]], vs[ts[:, 2]]))) / 6
    assert np.isclose(vol, 0.6 ** 3)                     # closed and outward
    key = lambda V: {tuple(sorted(tuple(np.round(V[i], 9)) for i in tr)) for tr in ts}
    ref = key(vs)
    for ax in range(3):
        w = vs.copy()
        w[:, ax] *= -1
        assert key(w) == ref                               # mirror-symmetric triangulation


def test_ellipsoid_workload():
    """Ellipsoid of the learned-preconditioner workload: semi-axes 4 x 2 x 1
    lambda0, eps 3 - 0.2j, 355 488 unknowns (edges about lambda0 / 28), every
    vertex on the ellipsoid, closed, outward, near-isotropic triangles,
    mirror-symmetric triangulation."""
    m = geo.workload("ellipsoid_c4")
    assert _unknowns(m) == 355488
    v, t = m["verts"], m["tris"]
    assert np.allclose(np.sum((v / [4.0, 2.0, 1.0]) ** 2, axis=1), 1.0)
    eps = m["media"][1, 0] + 1j * m["media"][1, 1]
    assert eps == 3.0 - 0.2j
    e = np.linalg.norm(v[t[:, [1, 2, 0]]] - v[t], axis=2)
    assert 0.03 < e.mean() < 0.04 and (e.max(1) / e.min(1)).max() < 2.5
    vol = np.sum(np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]]))) / 6
    assert abs(vol / (4 / 3 * np.pi * 8.0) - 1) < 1e-3
    s = geo.workload("ellipsoid_small")
    vs, ts = s["verts"], s["tris"]
    key = lambda V: {tuple(sorted(tuple(np.round(V[i], 9)) for i in tr)) for tr in ts}
    ref = key(vs)
    for ax in range(3):
        w = vs.copy()
        w[:, ax] *= -1
        assert key(w) == ref


def test_lens_on_slab_workload():
    """Three-layer lens on a slab (the multi-boundary body of Eq. 16), at the
    small size: every region's boundary is closed and consistently oriented,
    its enclosed volume is the body's (hemispheres to the mesh's chord error,
    the slab box exactly), region 0 encloses minus the whole body, and the
    junction edges are exactly the edges on the three base circles."""
    from oracle.rwg import Mesh
    radii, slab = (0.15, 0.3, 0.6), (1.4, 1.4, 0.2)
    g = geo.lens_on_slab(radii, slab=slab, nlon=24, h=0.1)
    v, t, reg = g["verts"], g["tris"], np.asarray(g["tri_regions"])
    trip = np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])) / 6
    hemi = [2.0 / 3.0 * np.pi * r ** 3 for r in (0.0,) + radii]
    want = [-(hemi[3] + slab[0] * slab[1] * slab[2])] + [hemi[k + 1] - hemi[k] for k in range(3)] \
        + [slab[0] * slab[1] * slab[2]]
    for l in range(5):
        on = (reg[:, 0] == l) | (reg[:, 1] == l)
        sgn = np.where(reg[on, 0] == l, -1.0, 1.0)          # the normal points into tri_regions[:, 0]
        vol = np.sum(sgn * trip[on])
        # inscribed hemispheres lose volume to the chord sag (edge / radius
        # about 0.7 on the inner layer here, 12 %): 15 % of the outer one; a
        # wrong side or material flips or moves whole layers (100 % and more)
        tol = 1e-12 if l == 4 else 0.15 * hemi[3 if l == 0 else l]
        assert abs(vol - want[l]) < tol, (l, vol, want[l])
        directed = {}
        for tr, s in zip(t[on], sgn):
            tr = tr if s > 0 else tr[::-1]
            for a, b in ((tr[0], tr[1]), (tr[1], tr[2]), (tr[2], tr[0])):
                directed[(a, b)] = directed.get((a, b), 0) + 1
        assert all(n == 1 and directed.get((b, a)) == 1 for (a, b), n in directed.items())
    m = Mesh(**g)
    va, vb = v[m.edge_v[:, 0]], v[m.edge_v[:, 1]]
    on_circle = np.zeros(m.ne, bool)
    for r in radii:
        on_circle |= (np.abs(va[:, 2]) < 1e-12) & (np.abs(vb[:, 2]) < 1e-12) \
            & (np.abs(np.hypot(va[:, 0], va[:, 1]) - r) < 1e-9) & (np.abs(np.hypot(vb[:, 0], vb[:, 1]) - r) < 1e-9)
    assert on_circle.sum() > 0 and np.array_equal(m.junction, on_circle)


def test_lens_on_slab_rejects_degenerate_bodies():
    """The generator refuses what it cannot mesh conformingly: point counts
    that do not put grid points on the slab's corners, layer radii out of
    order, a lens touching the slab's rim (the 6 lambda0 lens on a 12 lambda0
    square), and more points (nlon) than the outer base circle keeps at spacing
h (its ring would be halved below the nlon points of the blend to the rim)."""
    with pytest.raises(ValueError):
        geo.lens_on_slab((0.15, 0.3, 0.6), slab=(1.4, 1.4, 0.2), nlon=20, h=0.1)
    with pytest.raises(ValueError):
        geo.lens_on_slab((0.3, 0.15, 0.6), slab=(1.4, 1.4, 0.2), nlon=24, h=0.1)
    with pytest.raises(ValueError):
        geo.lens_on_slab((1.5, 3.0, 6.0), slab=(12.0, 12.0, 0.5), nlon=512, h=0.07)
    with pytest.raises(ValueError):
        geo.lens_on_slab((0.15, 0.3, 0.6), slab=(1.4, 1.4, 0.2), nlon=512, h=0.1)
    assert geo._ring_count(1.0, 0.1, 64) == 64          # spacing 0.098 at 64 points: no halving
    assert geo._ring_count(0.1, 0.1, 64) == 8           # 0.079 at 8 points; 4 would be below 5
    for n, m in ((8, 8), (8, 16)):
        tris = geo._band(list(range(n)), list(range(100, 100 + m)))
        assert len(tris) == n + m                        # every ring segment in exactly one triangle
    with pytest.raises(ValueError):
        geo._band(list(range(8)), list(range(24)))

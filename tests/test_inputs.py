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

"""Seeded synthetic inputs: triangulated dielectric bodies and excitation vectors.

This module generates *inputs* only (vertex/triangle arrays, region tables,
material tables, random coefficient vectors). It holds none of the solver's
arithmetic and is the one module shared by the CUDA path, its tests, the bench
and the CPU oracle.

Geometry conventions (the same ones the C ABI documents for ``sie_build_mesh``):

* ``verts``  float64 [nv, 3] in metres (lambda_0 = 1 m throughout).
* ``tris``   int32   [nt, 3]; the normal (v1-v0) x (v2-v0) points into
  ``tri_regions[t, 0]`` (the "+" region); ``tri_regions[t, 1]`` is the region
  behind the surface.
* ``media``  float64 [nr, 4] = (eps_r real, eps_r imag, mu_r real, mu_r imag);
  region 0 is the unbounded host medium that contains the sources.  Lossy media
  have eps_r imag < 0 (time convention exp(+j omega t)).

The bodies stand in for the paper's examples (single and multi-layer dielectric
spheres of Sect. "Simulation Results", Fig. 5); the paper's own meshes are not
published, so geodesic spheres of stated frequency are used.
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0          # speed of light [m/s]
LAMBDA0 = 1.0             # free-space wavelength of every synthetic case [m]
FREQ_HZ = C0 / LAMBDA0    # 299.792458 MHz


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def geodesic_sphere(nu: int, radius: float, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere of frequency ``nu``: 20 nu^2 triangles, 30 nu^2 edges,
    10 nu^2 + 2 vertices, every vertex on the sphere, normals pointing outward.
    nu = 8 gives the 1280-triangle / 1920-edge mesh of a level-3 icosphere."""
    if nu < 1:
        raise ValueError("nu must be >= 1")
    iv, faces = _icosahedron()
    # integer lattice keys make the vertex merge across faces exact
    key_to_idx: dict = {}
    pts = []
    tris = []
    # global lattice: a point is a + (b-a) i/nu + (c-a) j/nu; key it by the
    # exact barycentric combination over icosahedron vertex ids
    for (a, b, c) in faces:
        local = {}
        for i in range(nu + 1):
            for j in range(nu + 1 - i):
                k = nu - i - j
                comb = {}
                for vid, w in ((a, k), (b, i), (c, j)):
                    if w:
                        comb[vid] = comb.get(vid, 0) + w
                key = tuple(sorted(comb.items()))
                idx = key_to_idx.get(key)
                if idx is None:
                    p = (iv[a] * k + iv[b] * i + iv[c] * j) / nu
                    idx = len(pts)
                    key_to_idx[key] = idx
                    pts.append(p)
                local[(i, j)] = idx
        for i in range(nu):
            for j in range(nu - i):
                tris.append((local[(i, j)], local[(i + 1, j)], local[(i, j + 1)]))
                if i + j < nu - 1:
                    tris.append((local[(i + 1, j)], local[(i + 1, j + 1)], local[(i, j + 1)]))
    P = np.array(pts, dtype=np.float64)
    P = P / np.linalg.norm(P, axis=1, keepdims=True) * radius + np.asarray(center, np.float64)
    T = np.array(tris, dtype=np.int32)
    # orient outward
    c = P[T].mean(axis=1) - np.asarray(center)
    n = np.cross(P[T[:, 1]] - P[T[:, 0]], P[T[:, 2]] - P[T[:, 0]])
    flip = np.einsum("ij,ij->i", n, c) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return P, T


def homogeneous_sphere(nu=8, radius=0.5, eps_r=4.0, mu_r=1.0):
    """Single dielectric sphere in free space (one interface, two regions)."""
    v, t = geodesic_sphere(nu, radius)
    regions = np.tile(np.array([[0, 1]], np.int32), (len(t), 1))
    eps = complex(eps_r)
    media = np.array([[1.0, 0.0, 1.0, 0.0], [eps.real, eps.imag, mu_r, 0.0]], np.float64)
    return dict(verts=v, tris=t, tri_regions=regions, media=media)


def latlong_sphere(nlat: int, nlon: int, radius: float):
    """Sphere meshed on nlat latitude bands (even: the equator z = 0 is a ring
    of mesh edges) and nlon meridians; outward-oriented triangles.  Returns
    vertices, triangles and the vertex indices of the equator ring (in order
    of increasing longitude)."""
    if nlat % 2 or nlat < 2 or nlon < 3:
        raise ValueError("latlong_sphere: nlat must be even and >= 2, nlon >= 3")
    verts = [(0.0, 0.0, radius)]
    ring = []
    for i in range(1, nlat):
        th = np.pi * i / nlat
        row = []
        for j in range(nlon):
            ph = 2.0 * np.pi * j / nlon
            row.append(len(verts))
            verts.append((radius * np.sin(th) * np.cos(ph), radius * np.sin(th) * np.sin(ph), radius * np.cos(th)))
        ring.append(row)
    south = len(verts)
    verts.append((0.0, 0.0, -radius))
    tris = []
    for j in range(nlon):
        j1 = (j + 1) % nlon
        tris.append((0, ring[0][j], ring[0][j1]))
        for i in range(nlat - 2):
            a, b, c, d = ring[i][j], ring[i][j1], ring[i + 1][j], ring[i + 1][j1]
            tris.append((a, c, d))
            tris.append((a, d, b))
        tris.append((south, ring[-1][j1], ring[-1][j]))
    return np.array(verts, np.float64), np.array(tris, np.int32), np.array(ring[nlat // 2 - 1], np.int32)


def split_sphere(nlat=8, nlon=16, nrings=2, radius=0.3, eps_upper=4.0, eps_lower=4.0):
    """Dielectric sphere cut by the plane z = 0 into an upper region 1 and a
    lower region 2 (three surfaces: upper hemisphere 0|1, lower hemisphere
    0|2, the disk 1|2, meeting at the equator's junction edges).  The disk is
    meshed on nrings concentric rings of nlon points sharing the equator
    vertices; its normal +z points into region 1.  With eps_upper == eps_lower
    the body is the homogeneous sphere of the same outer mesh."""
    v, t, eq = latlong_sphere(nlat, nlon, radius)
    cen = v[:, 2]
    up = np.array([cen[list(tr)].mean() > 0 for tr in t])
    verts = [tuple(x) for x in v]
    rings = []
    for r in range(1, nrings):
        rho = radius * r / nrings
        row = []
        for j in range(nlon):
            ph = 2.0 * np.pi * j / nlon
            row.append(len(verts))
            verts.append((rho * np.cos(ph), rho * np.sin(ph), 0.0))
        rings.append(row)
    rings.append(list(eq))
    centre = len(verts)
    verts.append((0.0, 0.0, 0.0))
    disk = []
    for j in range(nlon):
        j1 = (j + 1) % nlon
        disk.append((centre, rings[0][j], rings[0][j1]))   # counter-clockwise seen from +z: normal +z
        for r in range(nrings - 1):
            a, b, c, d = rings[r][j], rings[r][j1], rings[r + 1][j], rings[r + 1][j1]
            disk.append((a, c, d))
            disk.append((a, d, b))
    tris = np.concatenate([t, np.array(disk, np.int32)])
    regions = np.concatenate([np.where(up[:, None], [[0, 1]], [[0, 2]]),
                              np.tile(np.array([[1, 2]]), (len(disk), 1))]).astype(np.int32)
    eu, el = complex(eps_upper), complex(eps_lower)
    media = np.array([[1, 0, 1, 0], [eu.real, eu.imag, 1, 0], [el.real, el.imag, 1, 0]], np.float64)
    return dict(verts=np.array(verts, np.float64), tris=tris, tri_regions=regions, media=media)


def latlong_homogeneous_sphere(nlat=8, nlon=16, radius=0.3, eps_r=4.0):
    """The outer surface of split_sphere as a single homogeneous body."""
    v, t, _ = latlong_sphere(nlat, nlon, radius)
    regions = np.tile(np.array([[0, 1]], np.int32), (len(t), 1))
    e = complex(eps_r)
    media = np.array([[1, 0, 1, 0], [e.real, e.imag, 1, 0]], np.float64)
    return dict(verts=v, tris=t, tri_regions=regions, media=media)


def _ring_count(rho, h, nmax):
    """Points on a ring of radius rho: nmax halved while the spacing stays
    below h (at least 5); nested rings keep each other's angles."""
    n = nmax
    while n % 2 == 0 and n // 2 >= 5 and 2.0 * np.pi * rho / (n // 2) <= h:
        n //= 2
    return n


def _band(inner, outer):
    """Triangles (vertex triples) between two nested rings with n and n or 2n
    points (angles increasing); orientation fixed by the caller."""
    n, m = len(inner), len(outer)
    out = []
    if m == n:
        for j in range(n):
            j1 = (j + 1) % n
            out += [(inner[j], outer[j], outer[j1]), (inner[j], outer[j1], inner[j1])]
    elif m == 2 * n:
        for j in range(n):
            j1 = (j + 1) % n
            b0, b1, b2 = outer[2 * j], outer[2 * j + 1], outer[(2 * j + 2) % m]
            out += [(inner[j], b0, b1), (inner[j], b1, inner[j1]), (inner[j1], b1, b2)]
    else:
        raise ValueError("_band: ring counts must be equal or double")
    return out


def lens_on_slab(radii=(1.5, 3.0, 6.0), eps_layers=(10.2, 4.5, 2.2), slab=(14.0, 14.0, 0.5), eps_slab=2.2,
                 nlon=256, h=0.15, nz=None):
    """Three-layer dielectric hemispherical lens on a dielectric slab (the
    multilayer body of the multi-boundary formulation, Eq. 16).  The lens
    layers are concentric hemispheres of the given radii resting on the slab's
    top face z = 0 (region 1 the innermost layer, eps_layers[0]; regions 2, 3
    the next; region 4 the slab, eps_slab, a box slab[0] x slab[1] x slab[2]
    below z = 0; region 0 free space).  The slab top is a polar grid whose
    rings include the three base circles (junction edges: a hemisphere, the
    top annulus inside it and the one outside meet there), blended from the
    outer circle to the slab's square rim; rings and hemisphere latitudes keep
    a spacing about h by halving their point counts toward the centre and the
    poles (nested angles, nlon at most; transition bands of three triangles);
    the bottom repeats the top grid; the side faces are rows at nz depths.
    nlon must be a multiple of 8 (the slab corners are grid points) and the
    slab must contain the base circle."""
    r1, r2, r3 = radii
    X, Y, T = slab[0] / 2.0, slab[1] / 2.0, slab[2]
    if nlon % 8 or not (0 < r1 < r2 < r3 < min(X, Y)):
        raise ValueError("lens_on_slab: nlon a multiple of 8 and radii increasing inside the slab")
    nz = nz or max(1, int(np.ceil(T / h)))
    verts = []

    def add(p):
        verts.append(p)
        return len(verts) - 1

    def ang(n):
        a = 2.0 * np.pi * np.arange(n) / n
        return np.cos(a), np.sin(a)

    # top grid ring radii (the base circles among them) and the material above each band
    radii_top, ring_mat = [], []
    lo = 0.0
    for k, rk in enumerate((r1, r2, r3)):
        n = max(1, int(np.ceil((rk - lo) / h)))
        for i in range(1, n + 1):
            radii_top.append(lo + (rk - lo) * i / n)
            ring_mat.append(k + 1)
        lo = rk
    counts = [_ring_count(rho, h, nlon) for rho in radii_top]
    for i in range(len(counts) - 2, -1, -1):      # at most a factor two between neighbours
        counts[i] = max(counts[i], counts[i + 1] // 2)
    n_rim = counts[-1]
    if n_rim != nlon:
        raise ValueError("lens_on_slab: nlon too large for h at the outer base circle")
    cr, sr = ang(nlon)
    tsq = np.minimum(X / np.maximum(np.abs(cr), 1e-300), Y / np.maximum(np.abs(sr), 1e-300))
    n_out = max(1, int(np.ceil((tsq.max() - r3) / h)))

    def top_grid(z):
        centre = add((0.0, 0.0, z))
        rings = []
        for rho, n in zip(radii_top, counts):
            c, s_ = ang(n)
            rings.append([add((rho * c[j], rho * s_[j], z)) for j in range(n)])
        for i in range(1, n_out + 1):
            t = i / n_out
            rings.append([add(((1 - t) * r3 * cr[j] + t * tsq[j] * cr[j],
                               (1 - t) * r3 * sr[j] + t * tsq[j] * sr[j], z)) for j in range(nlon)])
        return centre, rings

    ctop, rtop = top_grid(0.0)
    cbot, rbot = top_grid(-T)
    mats = ring_mat + [0] * n_out
    tris, regs = [], []

    def tri(a, b, c, want, reg):
        pa, pb, pc = (np.array(verts[q]) for q in (a, b, c))
        if np.dot(np.cross(pb - pa, pc - pa), want) < 0:
            b, c = c, b
        tris.append((a, b, c))
        regs.append(reg)

    up, down = np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0])
    for (cen, rings, want, top) in ((ctop, rtop, up, True), (cbot, rbot, down, False)):
        n0 = len(rings[0])
        for j in range(n0):
            tri(cen, rings[0][j], rings[0][(j + 1) % n0], want, (mats[0], 4) if top else (0, 4))
        for i in range(len(rings) - 1):
            for a, b, c in _band(rings[i], rings[i + 1]):
                tri(a, b, c, want, (mats[i + 1], 4) if top else (0, 4))
    # hemispheres: latitude rings from the base circle (shared with the top grid) to the pole
    cum = np.cumsum([max(1, int(np.ceil((rk - l0) / h))) for rk, l0 in ((r1, 0.0), (r2, r1), (r3, r2))])
    for k, rk in enumerate((r1, r2, r3)):
        base = rtop[cum[k] - 1]
        m = max(2, int(np.ceil(0.5 * np.pi * rk / h)))
        rings = [base]
        for i in range(1, m):
            th = 0.5 * np.pi * (1.0 - i / m)   # polar angle from +z
            n = max(_ring_count(rk * np.sin(th), h, len(base)), len(rings[-1]) // 2)
            c, s_ = ang(n)
            rings.append([add((rk * np.sin(th) * c[j], rk * np.sin(th) * s_[j], rk * np.cos(th))) for j in range(n)])
        pole = add((0.0, 0.0, rk))
        reg = (0 if k == 2 else k + 2, k + 1)
        for i in range(m - 1):
            for a, b, c in _band(rings[i + 1], rings[i]):
                cen = np.mean([verts[q] for q in (a, b, c)], axis=0)
                tri(a, b, c, cen, reg)
        nl = len(rings[-1])
        for j in range(nl):
            a, b = rings[-1][j], rings[-1][(j + 1) % nl]
            cen = np.mean([verts[q] for q in (a, b, pole)], axis=0)
            tri(a, b, pole, cen, reg)
    # side faces: rows below the square rim of the top grid down to the bottom grid's rim
    rim_t, rim_b = rtop[-1], rbot[-1]
    rows = [rim_t]
    for q in range(1, nz):
        z = -T * q / nz
        rows.append([add((verts[v][0], verts[v][1], z)) for v in rim_t])
    rows.append(rim_b)
    for j in range(nlon):
        j1 = (j + 1) % nlon
        pa, pb = np.array(verts[rim_t[j]]), np.array(verts[rim_t[j1]])
        mid = 0.5 * (pa + pb)
        want = np.array([np.sign(mid[0]) if abs(abs(mid[0]) - X) < 1e-9 else 0.0,
                         np.sign(mid[1]) if abs(abs(mid[1]) - Y) < 1e-9 else 0.0, 0.0])
        for q in range(nz):
            a, b, c, d = rows[q][j], rows[q][j1], rows[q + 1][j], rows[q + 1][j1]
            tri(a, c, d, want, (0, 4))
            tri(a, d, b, want, (0, 4))
    media = [[1.0, 0.0, 1.0, 0.0]]
    for e in list(eps_layers) + [eps_slab]:
        e = complex(e)
        media.append([e.real, e.imag, 1.0, 0.0])
    return dict(verts=np.array(verts, np.float64), tris=np.array(tris, np.int32),
                tri_regions=np.array(regs, np.int32), media=np.array(media, np.float64))


def coated_sphere(nu_outer=30, nu_inner=20, r_outer=1.5, r_inner=1.0, eps_shell=2.56, eps_core=4.0):
    """Two-layer sphere: region 0 free space, region 1 shell, region 2 core."""
    vo, to = geodesic_sphere(nu_outer, r_outer)
    vi, ti = geodesic_sphere(nu_inner, r_inner)
    verts = np.concatenate([vo, vi])
    tris = np.concatenate([to, ti + len(vo)]).astype(np.int32)
    regions = np.concatenate([np.tile([[0, 1]], (len(to), 1)), np.tile([[1, 2]], (len(ti), 1))]).astype(np.int32)
    es, ec = complex(eps_shell), complex(eps_core)
    media = np.array([[1, 0, 1, 0], [es.real, es.imag, 1, 0], [ec.real, ec.imag, 1, 0]], np.float64)
    return dict(verts=verts, tris=tris, tri_regions=regions, media=media)


def tetra_body(size=0.3, eps_r=4.0):
    """Tiny closed body (4 triangles, 6 edges) for brute-force checks."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64) * size
    t = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    regions = np.tile(np.array([[0, 1]], np.int32), (4, 1))
    media = np.array([[1, 0, 1, 0], [eps_r, 0, 1, 0]], np.float64)
    return dict(verts=v, tris=t, tri_regions=regions, media=media)


def cube_surface(n: int, side: float, center=(0.0, 0.0, 0.0)):
    """Closed cube surface of edge ``side`` on a structured grid of n x n
    squares per face, each square cut into two right triangles: 12 n^2
    triangles, 18 n^2 edges, 6 n^2 + 2 vertices, normals pointing outward.
    Vertices are merged across faces by exact integer lattice keys.  The
    diagonal of each square leans one way in the lower half of a face and
    the other way in the upper half (with respect to each in-plane axis), so
    for even n the triangulation is mirror-symmetric under x -> -x, y -> -y
    and z -> -z (the mirror images of the RCS are exact symmetries of the
    discrete problem, not only of the body)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    key_to_idx: dict = {}
    pts = []
    tris = []

    def vid(ijk):
        idx = key_to_idx.get(ijk)
        if idx is None:
            idx = len(pts)
            key_to_idx[ijk] = idx
            pts.append(ijk)
        return idx

    h = n / 2.0
    for axis in range(3):
        a1, a2 = (axis + 1) % 3, (axis + 2) % 3
        for side_sign in (0, n):
            for i in range(n):
                for j in range(n):
                    def corner(di, dj):
                        p = [0, 0, 0]
                        p[axis] = side_sign
                        p[a1] = i + di
                        p[a2] = j + dj
                        return vid(tuple(p))
                    v00, v10, v01, v11 = corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)
                    # lean of the diagonal mirrors about the face's centre lines
                    if (i + 0.5 < h) == (j + 0.5 < h):
                        tris.append((v00, v10, v11))
                        tris.append((v00, v11, v01))
                    else:
                        tris.append((v00, v10, v01))
                        tris.append((v10, v11, v01))
    P = (np.array(pts, dtype=np.float64) / n - 0.5) * side + np.asarray(center, np.float64)
    T = np.array(tris, dtype=np.int32)
    c = P[T].mean(axis=1) - np.asarray(center)
    nrm = np.cross(P[T[:, 1]] - P[T[:, 0]], P[T[:, 2]] - P[T[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, c) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return P, T


def box_surface(nx: int, ny: int, nz: int):
    """Closed surface of the cube [-1, 1]^3 on a structured grid with nx, ny,
    nz divisions along x, y, z, each rectangle cut into two triangles whose
    diagonals mirror about the faces' centre lines (as in cube_surface):
    4 (nx ny + ny nz + nz nx) triangles, outward normals."""
    n = (nx, ny, nz)
    key_to_idx: dict = {}
    pts = []
    tris = []

    def vid(ijk):
        idx = key_to_idx.get(ijk)
        if idx is None:
            idx = len(pts)
            key_to_idx[ijk] = idx
            pts.append(ijk)
        return idx

    for axis in range(3):
        a1, a2 = (axis + 1) % 3, (axis + 2) % 3
        for side_sign in (0, n[axis]):
            for i in range(n[a1]):
                for j in range(n[a2]):
                    def corner(di, dj):
                        p = [0, 0, 0]
                        p[axis] = side_sign
                        p[a1] = i + di
                        p[a2] = j + dj
                        return vid(tuple(p))
                    v00, v10, v01, v11 = corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)
                    if (2 * i + 1 < n[a1]) == (2 * j + 1 < n[a2]):
                        tris.append((v00, v10, v11))
                        tris.append((v00, v11, v01))
                    else:
                        tris.append((v00, v10, v01))
                        tris.append((v10, v11, v01))
    P = 2.0 * np.array(pts, dtype=np.float64) / np.array(n, dtype=np.float64) - 1.0
    T = np.array(tris, dtype=np.int32)
    c = P[T].mean(axis=1)
    nrm = np.cross(P[T[:, 1]] - P[T[:, 0]], P[T[:, 2]] - P[T[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, c) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return P, T


def ellipsoid_surface(m: int, axes=(4.0, 2.0, 1.0)):
    """Tri-axial ellipsoid with semi-axes (a, b, c), a >= b >= c, by the
    cube-sphere mapping: the surface of [-1, 1]^3 with divisions proportional
    to the semi-axes (m a / c, m b / c, m along x, y, z) is projected radially
    onto the unit sphere and scaled by the semi-axes, which keeps the
    triangles near-isotropic.  Every vertex lies on the ellipsoid; outward
    normals.  4 m^2 (ab + bc + ca) / c^2 triangles."""
    a, b, c = (float(v) for v in axes)
    nx, ny, nz = int(round(m * a / c)), int(round(m * b / c)), int(m)
    P, T = box_surface(nx, ny, nz)
    U = P / np.linalg.norm(P, axis=1, keepdims=True)
    V = U * np.array([a, b, c])
    ctr = V[T].mean(axis=1)
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, ctr) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return V, T


def dielectric_ellipsoid(m=46, axes=(4.0, 2.0, 1.0), eps_r=3.0 - 0.2j, mu_r=1.0):
    """Homogeneous (lossy) dielectric ellipsoid in free space, one interface."""
    v, t = ellipsoid_surface(m, axes)
    regions = np.tile(np.array([[0, 1]], np.int32), (len(t), 1))
    eps = complex(eps_r)
    media = np.array([[1.0, 0.0, 1.0, 0.0], [eps.real, eps.imag, mu_r, 0.0]], np.float64)
    return dict(verts=v, tris=t, tri_regions=regions, media=media)


def dielectric_cube(n=54, side=3.0, eps_r=6.0 - 0.6j, mu_r=1.0):
    """Homogeneous (lossy) dielectric cube in free space, one interface."""
    v, t = cube_surface(n, side)
    regions = np.tile(np.array([[0, 1]], np.int32), (len(t), 1))
    eps = complex(eps_r)
    media = np.array([[1.0, 0.0, 1.0, 0.0], [eps.real, eps.imag, mu_r, 0.0]], np.float64)
    return dict(verts=v, tris=t, tri_regions=regions, media=media)


# Plasmonic coated nanoparticle: silver-like core in a gold-like shell at
# 545 THz (lambda0 = 550 nm).  Assumed round permittivities with negative real
# parts and loss (e^{+jwt}: eps'' < 0), of the size of noble-metal data at
# that wavelength; not tabulated measurements.
NANO_EPS_CORE = -10.0 - 0.8j
NANO_EPS_SHELL = -5.0 - 2.0j


# Named workloads (sizes follow the configurations the solver is measured on)
def workload(name: str):
    if name == "sphere_c1":      # radius 0.5 lambda0, eps 4, 1280 tri, 3840 unknowns
        return homogeneous_sphere(nu=8, radius=0.5, eps_r=4.0)
    if name == "coated_c2":      # 1.0/1.5 lambda0, eps 4/2.56, ~78k unknowns
        return coated_sphere(30, 20)
    if name == "coated_small":   # reduced coated sphere, ~12.5k unknowns
        return coated_sphere(12, 8)
    if name == "nanoparticle":   # plasmonic coated sphere (core 230, shell 250 at 550 nm), 30 720 unknowns
        return coated_sphere(16, 16, 250 / 550, 230 / 550, NANO_EPS_SHELL, NANO_EPS_CORE)
    if name == "cube_c3":        # cube 3 lambda0, eps 6 - 0.6j, 54 x 54 squares per face, 104 976 unknowns
        return dielectric_cube(54, 3.0, 6.0 - 0.6j)
    if name == "cube_small":     # same material, 0.6 lambda0, 14 x 14 squares per face: dense CPU checks
        return dielectric_cube(14, 0.6, 6.0 - 0.6j)
    if name == "cube_tiny":      # same material, 0.6 lambda0, 6 x 6 squares per face
        return dielectric_cube(6, 0.6, 6.0 - 0.6j)
    if name == "ellipsoid_c4":   # semi-axes 4 x 2 x 1 lambda0, eps 3 - 0.2j, 355 488 unknowns
        return dielectric_ellipsoid(46, (4.0, 2.0, 1.0), 3.0 - 0.2j)
    if name == "ellipsoid_small":  # semi-axes 1.0 x 0.5 x 0.25 lambda0, same material: dense CPU checks
        return dielectric_ellipsoid(4, (1.0, 0.5, 0.25), 3.0 - 0.2j)
    if name == "lens_c5":        # 3-layer lens (radii 1.5/3/6, eps 10.2/4.5/2.2) on a 14 x 14 x 0.5 slab (eps 2.2), 1 189 264 unknowns
        return lens_on_slab((1.5, 3.0, 6.0), (10.2, 4.5, 2.2), (14.0, 14.0, 0.5), 2.2, nlon=512, h=0.07)
    if name == "lens_small":     # the same body at 0.1 scale: dense CPU checks
        return lens_on_slab((0.15, 0.3, 0.6), slab=(1.4, 1.4, 0.2), nlon=24, h=0.1)
    if name == "coated_tiny":    # coated sphere small enough for dense CPU checks
        return coated_sphere(6, 4)
    if name == "sphere_tiny":
        return homogeneous_sphere(nu=3, radius=0.5, eps_r=4.0)
    raise KeyError(name)


def random_coefficients(n_unknowns: int, nrhs: int = 1, seed: int = 1234):
    """Complex standard-normal coefficient vectors, shape [nrhs, n_unknowns]."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((nrhs, n_unknowns)) + 1j * rng.standard_normal((nrhs, n_unknowns))) / np.sqrt(2.0)
    return x.astype(np.complex128)


def bistatic_angles(n=361):
    """Observation angles theta in [0, 180] deg in the phi = 0 plane, as (theta, phi) radians."""
    th = np.linspace(0.0, np.pi, n)
    return np.stack([th, np.zeros_like(th)], axis=1)


def monostatic_incidences(n, seed=None):
    """Incidence list rows (theta_i, phi_i, pol_angle, E0): theta uniform in [0, pi], phi = 0, theta-pol."""
    th = np.linspace(0.0, np.pi, n)
    return np.stack([th, np.zeros(n), np.zeros(n), np.ones(n)], axis=1)

"""RWG basis functions on a multi-region triangulation (oracle, test infrastructure).

Follows Eq. 22 and Fig. 4 of the paper: one basis per interior edge of an
interface surface, supported on the two triangles T+ and T- sharing it,

    f(r) = +l/(2A+) (r - v+)   on T+,      f(r) = -l/(2A-) (r - v-)   on T-,

with v+/- the free (non-edge) vertices; div f = +l/A+ on T+ and -l/A- on T-.

Ordering rule (shared by definition with the C ABI, written independently
here): an edge is the unordered vertex pair of a triangle side; edges owned by
exactly two triangles are RWG edges; they are numbered in lexicographic order
of (min vertex, max vertex); T+ is the owning triangle with the smaller index.
Multi-region tables (Eqs. 12-13): the surface normal of a triangle points into
tri_regions[t, 0].  For region l, an edge on a surface with "+" region l has
sign s_l = +1; with "-" region l, s_l = -1; otherwise the edge is not in B_l.

Junction edges (Eq. 16's multi-boundary setting where three or more surfaces
meet at an edge; the paper's multilayer bodies): each region l that touches
the edge sees exactly two of its triangles, T1 and T2, and region l's
equivalent current n_l x H has a continuous normal component across the edge
within its own boundary (it is -H.t on both faces, whatever the wedge angle).
With the currents of a face shared by two regions equal and opposite, the
currents of all faces at the edge are then tied to one unknown (one for J,
one for M): on triangle T the surface current crossing the edge is
a_T u h_T, where h_T is the RWG half-function of T (flowing out of T across
the edge), and for every region l touching the edge
    s_l(T1) a_T1 = - s_l(T2) a_T2,
s_l(T) = +1 if l is the "+" region of T and -1 otherwise.  Around the edge
these constraints are consistent (each face is counted once by each of its
two regions).  Region l's basis function is then s_l(T1) a_T1 (h_T1 - h_T2),
an RWG function on T1, T2.  An ordinary edge is the case of two triangles of
one surface with a_T+ = +1, a_T- = -1.  The tables below store a_T per
triangle side (tri_sign); the region's sign s_l(T) enters per triangle.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, verts, tris, tri_regions, media):
        self.verts = np.asarray(verts, np.float64)
        self.tris = np.asarray(tris, np.int64)
        self.tri_regions = np.asarray(tri_regions, np.int64)
        self.media = np.asarray(media, np.float64)
        self.nt = len(self.tris)
        self.nr = len(self.media)
        P = self.verts[self.tris]                       # [nt,3,3]
        cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.normal = cr / (2.0 * self.area[:, None])
        self.centroid = P.mean(axis=1)
        self.hmax = np.max(np.linalg.norm(P - np.roll(P, -1, axis=1), axis=2), axis=1)
        self._build_edges()

    def _build_edges(self):
        owners = {}
        for t in range(self.nt):
            a, b, c = (int(x) for x in self.tris[t])
            for (u, v, w) in ((a, b, c), (b, c, a), (c, a, b)):
                key = (min(u, v), max(u, v))
                owners.setdefault(key, []).append((t, w, (u, v)))
        keys = sorted(k for k, o in owners.items() if len(o) >= 2)
        ne = len(keys)
        self.ne = ne
        self.edge_v = np.array(keys, np.int64).reshape(ne, 2)
        self.tp = np.zeros(ne, np.int64)
        self.tm = np.zeros(ne, np.int64)
        self.vp = np.zeros(ne, np.int64)     # free vertex of T+
        self.vm = np.zeros(ne, np.int64)     # free vertex of T-
        # local edge table per triangle: (rwg index or -1, sign, free vertex)
        self.tri_edge = -np.ones((self.nt, 3), np.int64)
        self.tri_sign = np.zeros((self.nt, 3), np.float64)
        self.tri_free = np.zeros((self.nt, 3), np.int64)
        self.junction = np.zeros(ne, bool)
        fill = np.zeros(self.nt, np.int64)
        for i, key in enumerate(keys):
            own = sorted(owners[key], key=lambda o: o[0])
            if len(own) == 2:
                (t1, w1, d1), (t2, w2, d2) = own
                if tuple(self.tri_regions[t1]) != tuple(self.tri_regions[t2]):
                    raise ValueError("edge shared by triangles of different surfaces")
                if d1 != (d2[1], d2[0]):
                    raise ValueError("inconsistent triangle orientation across an edge")
                sides = ((t1, w1, 1.0), (t2, w2, -1.0))
            else:
                sides = self._junction_signs(own)
                self.junction[i] = True
                (t1, w1, _), (t2, w2, _) = own[0], own[1]
            self.tp[i], self.vp[i], self.tm[i], self.vm[i] = t1, w1, t2, w2
            for t, w, s in sides:
                j = fill[t]
                self.tri_edge[t, j] = i
                self.tri_sign[t, j] = s
                self.tri_free[t, j] = w
                fill[t] += 1
        self.length = np.linalg.norm(self.verts[self.edge_v[:, 1]] - self.verts[self.edge_v[:, 0]], axis=1)
        self.edge_mid = 0.5 * (self.verts[self.edge_v[:, 0]] + self.verts[self.edge_v[:, 1]])
        self.edge_regions = self.tri_regions[self.tp]     # (r+, r-)

    def _junction_signs(self, own):
        """Coefficients a_T of the triangles meeting at a junction edge (see the
        module docstring): a_T of the first triangle is +1, the others follow
        from s_l(T1) a_T1 = -s_l(T2) a_T2 for each region l touching the edge.
        Raises when a region sees other than two of the triangles or when the
        constraints do not close."""
        tris = [t for t, _, _ in own]
        regs = sorted({int(r) for t in tris for r in self.tri_regions[t]})
        pairs = []
        for l in regs:
            tl = [t for t in tris if l in self.tri_regions[t]]
            if len(tl) != 2:
                raise ValueError(f"junction edge: region {l} sees {len(tl)} of its triangles (need 2)")
            pairs.append((l, tl[0], tl[1]))
        sl = lambda l, t: 1.0 if self.tri_regions[t, 0] == l else -1.0
        a = {tris[0]: 1.0}
        for _ in range(len(pairs)):
            for l, t1, t2 in pairs:
                if t1 in a and t2 not in a:
                    a[t2] = -sl(l, t1) * sl(l, t2) * a[t1]
                elif t2 in a and t1 not in a:
                    a[t1] = -sl(l, t1) * sl(l, t2) * a[t2]
        if len(a) != len(tris):
            raise ValueError("junction edge: triangles not connected through the regions")
        for l, t1, t2 in pairs:
            if sl(l, t1) * a[t1] != -sl(l, t2) * a[t2]:
                raise ValueError("junction edge: inconsistent current continuity constraints")
        return tuple((t, w, a[t]) for t, w, _ in own)

    # ---- per-region tables (Eqs. 12-13) ----
    def region_sign(self, l):
        """s_l(n) for every edge: +1 / -1 / 0 (edge not on the boundary of B_l).
        Not defined for junction edges (their sign is per triangle)."""
        s = np.zeros(self.ne)
        s[self.edge_regions[:, 0] == l] = 1.0
        s[self.edge_regions[:, 1] == l] = -1.0
        return s

    def region_tris(self, l):
        return np.nonzero((self.tri_regions[:, 0] == l) | (self.tri_regions[:, 1] == l))[0]

    def tri_region_sign(self, l):
        s = np.zeros(self.nt)
        s[self.tri_regions[:, 0] == l] = 1.0
        s[self.tri_regions[:, 1] == l] = -1.0
        return s


def material(media_row, k0):
    """k_l = k0 sqrt(eps_r mu_r) with Im k <= 0 and relative impedance
    eta_l / eta_0 = sqrt(mu_r / eps_r) with Re > 0 (Eq. 7 definitions, e^{+j w t})."""
    eps = complex(media_row[0], media_row[1])
    mu = complex(media_row[2], media_row[3])
    k = k0 * np.sqrt(eps * mu)          # principal root: Re k >= 0, Im k <= 0 for passive media
    if k.imag > 0:
        raise ValueError("active medium (Im eps_r mu_r > 0) is not supported")
    eta = np.sqrt(mu / eps)
    if eta.real < 0:
        eta = -eta
    return complex(k), complex(eta)

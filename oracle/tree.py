"""Octree box assignment, near-field pattern and preconditioner ordering
(oracle copy, test infrastructure; the library implements the same rule
independently).

The paper gives no MLFMM or ILU details (it cites them); the definitions used
by both sides are:

* root cube: centre = midpoint of the vertex bounding box, edge
  D = (largest bounding-box extent) * 1.0009765625; ``nlev`` levels, leaf edge
  h = D / 2^(nlev-1).
* an RWG basis belongs to the leaf box containing its edge midpoint
  0.5 (va + vb): i = floor((x - (centre - D/2)) / h), clamped to the grid.
* near pattern: basis pairs whose leaf boxes touch (|di|,|dj|,|dk| <= 1).
* ILU ordering: leaf boxes coloured by coordinate parity
  colour = (i&1) | (j&1)<<1 | (k&1)<<2 (touching boxes never share a colour);
  bases sorted by (colour, Morton code of the box, edge index).
"""
from __future__ import annotations

import numpy as np


def box_coords(mesh, nlev):
    lo = mesh.verts.min(axis=0)
    hi = mesh.verts.max(axis=0)
    centre = (lo + hi) * 0.5
    D = float(np.max(hi - lo)) * 1.0009765625
    origin = centre - 0.5 * D
    nleaf = 1 << (nlev - 1)
    h = D / nleaf
    mid = (mesh.verts[mesh.edge_v[:, 0]] + mesh.verts[mesh.edge_v[:, 1]]) * 0.5
    ijk = np.floor((mid - origin) / h).astype(np.int64)
    return np.clip(ijk, 0, nleaf - 1)


def morton(ijk):
    code = np.zeros(len(ijk), np.int64)
    for b in range(21):
        for a in range(3):
            code |= ((ijk[:, a] >> b) & 1) << (3 * b + a)
    return code


def colour(ijk):
    return (ijk[:, 0] & 1) | ((ijk[:, 1] & 1) << 1) | ((ijk[:, 2] & 1) << 2)


def ordering(mesh, nlev):
    """perm[p] = edge index at internal position p."""
    ijk = box_coords(mesh, nlev)
    keys = np.lexsort((np.arange(mesh.ne), morton(ijk), colour(ijk)))
    return keys


def near_mask(mesh, nlev):
    """Dense boolean [ne, ne]: True where the leaf boxes of m and n touch."""
    ijk = box_coords(mesh, nlev)
    d = np.abs(ijk[:, None, :] - ijk[None, :, :]).max(axis=2)
    return d <= 1

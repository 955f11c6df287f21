"""Triangle quadrature rules (oracle copy; the CUDA library holds its own).

* ``radon7``: Radon's 7-point degree-5 symmetric rule (a published rule; the
  same rule is used by the library for every regular integral so that the
  two sides discretise identically).
* ``collapsed_gauss(n)``: n x n Gauss-Legendre product rule mapped to the
  triangle by the collapsed (Duffy) map, exact to polynomial degree 2n-2.
  Used as the outer rule of singular / near-singular triangle pairs.

Rules are returned in barycentric form (b [q,3], w [q]) with sum(w) = 1, so
that  int_T f dA ~= A * sum_q w_q f(sum_i b_qi v_i).
"""
from __future__ import annotations

import numpy as np


def radon7():
    s = np.sqrt(15.0)
    a1, a2 = (6.0 - s) / 21.0, (6.0 + s) / 21.0
    w1, w2 = (155.0 - s) / 1200.0, (155.0 + s) / 1200.0
    b = [(1 / 3, 1 / 3, 1 / 3)]
    w = [9.0 / 40.0]
    for a, wt in ((a1, w1), (a2, w2)):
        c = 1.0 - 2.0 * a
        b += [(c, a, a), (a, c, a), (a, a, c)]
        w += [wt, wt, wt]
    return np.array(b, np.float64), np.array(w, np.float64)


def collapsed_gauss(n: int):
    x, wx = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (x + 1.0)
    wu = 0.5 * wx
    bs, ws = [], []
    for i in range(n):
        for j in range(n):
            xi = u[i]
            eta = u[j] * (1.0 - u[i])
            bs.append((1.0 - xi - eta, xi, eta))
            ws.append(2.0 * wu[i] * wu[j] * (1.0 - u[i]))
    return np.array(bs, np.float64), np.array(ws, np.float64)


def points(tri_verts, b):
    """tri_verts [..., 3, 3] -> quadrature points [..., q, 3]."""
    return np.einsum("qi,...ix->...qx", b, tri_verts)

"""Linear solvers (oracle, test infrastructure).

* ``lu_solve``: dense LU with partial pivoting (LAPACK zgesv via numpy).
* ``fgmres``: restarted flexible GMRES(m) with right preconditioning (Saad,
  Iterative Methods for Sparse Linear Systems, Alg. 9.6), modified
  Gram-Schmidt, complex Givens rotations.  The paper solves with
  ILU-preconditioned BiCGStab; the measured workload uses GMRES(50) with the
  same ILU (the reading adopted for the solver choice).
* ``bicgstab``: BiCGStab (van der Vorst 1992) and ``cgs``: conjugate
  gradient squared (Sonneveld 1989), right-preconditioned, with the complex
  inner product (a, b) = sum conj(a) b; the paper's solvers (its iteration
  study compares ILU-BiCGStab, CGS and GMRES).  Iterations count steps, each
  with two products and two preconditioner applications.
* ``ilu0``: incomplete LU with zero fill on a given sparsity pattern (the
  paper's ILU preconditioner, cited without detail): L unit lower, U upper,
  (L U)_ij = A_ij for every (i, j) of the pattern; IKJ elimination order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


def lu_solve(Z, b):
    return np.linalg.solve(Z, np.asarray(b).T).T


def fgmres(matvec, b, precond=None, restart=50, tol=1e-4, maxit=2000, x0=None):
    """Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, np.complex128)
    n = b.shape[0]
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    its = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm < tol or its >= maxit:
            return x, its, hist
        V = np.zeros((restart + 1, n), np.complex128)
        Zs = np.zeros((restart, n), np.complex128)
        H = np.zeros((restart + 1, restart), np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, np.complex128)
        g = np.zeros(restart + 1, np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(restart):
            z = precond(V[j]) if precond is not None else V[j]
            Zs[j] = z
            w = matvec(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            if bb == 0:
                c, s = 1.0, 0.0
            elif a == 0:
                c, s = 0.0, 1.0
            else:
                t = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
                c = abs(a) / t
                s = (a / abs(a)) * np.conj(bb) / t
            cs[j], sn[j] = c, s
            H[j, j] = c * a + s * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            its += 1
            j_end = j + 1
            if abs(g[j + 1]) / bnorm < tol or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Zs[:j_end].T @ y


def bicgstab(matvec, b, precond=None, tol=1e-4, maxit=2000, x0=None):
    """Right-preconditioned BiCGStab: solves A M^-1 u = b, x = M^-1 u, with
    shadow residual r0.  Returns (x, iterations, relative residual history)."""
    M = precond if precond is not None else (lambda v: v)
    b = np.asarray(b, np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    r = b - matvec(x)
    rs = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = [np.linalg.norm(r) / bnorm]
    its = 0
    while hist[-1] >= tol and its < maxit:
        rho_new = np.vdot(rs, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = matvec(ph)
        alpha = rho_new / np.vdot(rs, v)
        s_ = r - alpha * v
        its += 1
        if np.linalg.norm(s_) / bnorm < tol:
            x = x + alpha * ph
            hist.append(np.linalg.norm(s_) / bnorm)
            break
        sh = M(s_)
        t = matvec(sh)
        omega = np.vdot(t, s_) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s_ - omega * t
        rho = rho_new
        hist.append(np.linalg.norm(r) / bnorm)
    return x, its, hist


def cgs(matvec, b, precond=None, tol=1e-4, maxit=2000, x0=None):
    """Right-preconditioned conjugate gradient squared with shadow residual r0.
    Returns (x, iterations, relative residual history)."""
    M = precond if precond is not None else (lambda v: v)
    b = np.asarray(b, np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    r = b - matvec(x)
    rs = r.copy()
    q = np.zeros_like(b)
    p = np.zeros_like(b)
    rho_old = 1.0 + 0j
    hist = [np.linalg.norm(r) / bnorm]
    its = 0
    while hist[-1] >= tol and its < maxit:
        rho = np.vdot(rs, r)
        if its == 0:
            u = r.copy()
            p = u.copy()
        else:
            beta = rho / rho_old
            u = r + beta * q
            p = u + beta * (q + beta * p)
        vh = matvec(M(p))
        alpha = rho / np.vdot(rs, vh)
        q = u - alpha * vh
        uh = M(u + q)
        x = x + alpha * uh
        r = r - alpha * matvec(uh)
        rho_old = rho
        its += 1
        hist.append(np.linalg.norm(r) / bnorm)
    return x, its, hist


def pattern_matrix(Z, mask_edges, perm):
    """Near-field matrix in the preconditioner ordering, as CSR over scalar
    unknowns: edge pattern ``mask_edges`` [ne, ne] expanded to 2x2 blocks,
    rows/cols permuted so that internal position p holds edge perm[p]."""
    ne = len(perm)
    inv = np.empty(ne, np.int64)
    inv[perm] = np.arange(ne)
    ii, jj = np.nonzero(mask_edges)
    rows, cols, vals = [], [], []
    for a in range(2):
        for c in range(2):
            rows.append(2 * inv[ii] + a)
            cols.append(2 * inv[jj] + c)
            vals.append(Z[2 * ii + a, 2 * jj + c])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(2 * ne, 2 * ne))
    A.sort_indices()
    return A


def ilu0(A: sp.csr_matrix):
    """ILU(0) of a CSR matrix (sorted indices, diagonal present).  Returns the
    combined factor in the pattern of A (strict lower part = L, upper = U)."""
    A = A.tocsr(copy=True)
    A.sort_indices()
    n = A.shape[0]
    ip, ix, d = A.indptr, A.indices, A.data
    diag = np.empty(n, np.int64)
    for i in range(n):
        pos = np.searchsorted(ix[ip[i]:ip[i + 1]], i)
        if pos >= ip[i + 1] - ip[i] or ix[ip[i] + pos] != i:
            raise ValueError("missing diagonal")
        diag[i] = ip[i] + pos
    where = -np.ones(n, np.int64)
    for i in range(n):
        s, e = ip[i], ip[i + 1]
        where[ix[s:e]] = np.arange(e - s)
        for kk in range(s, diag[i]):
            k = ix[kk]
            d[kk] = d[kk] / d[diag[k]]
            ks, ke = diag[k] + 1, ip[k + 1]
            w = where[ix[ks:ke]]
            ok = w >= 0
            d[s + w[ok]] -= d[kk] * d[ks:ke][ok]
        where[ix[s:e]] = -1
    return A


def ilu_apply(F: sp.csr_matrix, v):
    """z = U^-1 L^-1 v for the combined ILU(0) factor F."""
    n = F.shape[0]
    Lm = sp.tril(F, k=-1, format="csr") + sp.identity(n, dtype=F.dtype, format="csr")
    Um = sp.triu(F, k=0, format="csr")
    y = spsolve_triangular(Lm, v, lower=True, unit_diagonal=True)
    return spsolve_triangular(Um, y, lower=False)

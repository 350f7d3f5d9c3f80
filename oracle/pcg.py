"""CPU oracle of the preconditioned conjugate-gradient loop -- TEST
INFRASTRUCTURE (only tests, smoke() and the benchmark's CPU legs use it).

The triangular solve is the kernel of preconditioners such as symmetric
Gauss-Seidel (the paper's Sec. I names iterative solvers as the consumers of
SpTRSV).  This module writes out, in FP64 and in the textbook order:

* ``sgs_apply``   z = M^{-1} r for M = (D + L) D^{-1} (D + L)^T, the symmetric
  Gauss-Seidel preconditioner of an SPD matrix A = L + D + L^T: a forward
  substitution with the lower triangle (D + L), a scaling by D, a backward
  substitution with (D + L)^T -- each by the oracle's own substitutions;
* ``pcg``          preconditioned conjugate gradients (Hestenes-Stiefel form):
  r0 = b - A x0, z0 = M^{-1} r0, p0 = z0; per step alpha = (r, z) / (p, A p),
  x += alpha p, r -= alpha A p, stop when |r|_2 <= rtol |b|_2, z = M^{-1} r,
  beta = (r_new, z_new) / (r, z), p = z + beta p.

Parity status: pinned by tests against a dense solve, the dense M^{-1}, and
CG's property of reaching the solution of an n-dimensional system in at most
n steps (up to rounding) on small matrices.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import backward_subst, forward_subst, transpose


def _spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x by scipy's CSR product (a library primitive)."""
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)) @ x


def lower_triangle(A):
    """D + L of a CSR A (entries with column <= row), as a CSR."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    keep = A.col <= rows
    cnt = np.bincount(rows[keep], minlength=A.n)
    ptr = np.zeros(A.n + 1, np.int64)
    np.cumsum(cnt, out=ptr[1:])
    return type(A)(A.n, ptr.astype(np.int32), A.col[keep].astype(np.int32),
                   np.ascontiguousarray(A.val[keep]))


def sgs_apply(Lo, r: np.ndarray) -> np.ndarray:
    """z = ((D + L) D^{-1} (D + L)^T)^{-1} r with Lo = D + L."""
    y = forward_subst(Lo, r)
    d = Lo.val[Lo.row_ptr[1:] - 1]          # the diagonal, last in every row
    return backward_subst(transpose(Lo), d * y)


def pcg(A, b: np.ndarray, x0: np.ndarray, rtol: float, max_iter: int):
    """(x, iterations, |r|_2 / |b|_2) of preconditioned CG with the symmetric
    Gauss-Seidel preconditioner built from A's lower triangle."""
    Lo = lower_triangle(A)
    x = np.array(x0, dtype=np.float64)
    r = b - _spmv(A, x)
    bnorm = float(np.sqrt(np.dot(b, b)))
    z = sgs_apply(Lo, r)
    p = z.copy()
    rz = float(np.dot(r, z))
    it = 0
    rel = float(np.sqrt(np.dot(r, r))) / bnorm
    while it < max_iter and rel > rtol:
        q = _spmv(A, p)
        alpha = rz / float(np.dot(p, q))
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.sqrt(np.dot(r, r))) / bnorm
        if rel <= rtol:
            break
        z = sgs_apply(Lo, r)
        rz_new = float(np.dot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel

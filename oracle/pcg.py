"""CPU oracle of the preconditioned conjugate-gradient loop -- TEST
INFRASTRUCTURE (only tests, smoke() and the benchmark's CPU legs use it).

The triangular solve is the kernel of preconditioners such as symmetric
Gauss-Seidel (the paper's Sec. I names iterative solvers as the consumers of
SpTRSV).  This module writes out, in FP64 and in the textbook order:

* ``sgs_apply``   z = M^{-1} r for M = (D + L) D^{-1} (D + L)^T, the symmetric
  Gauss-Seidel preconditioner of an SPD matrix A = L + D + L^T: a forward
  substitution with the lower triangle (D + L), a scaling by D, a backward
  substitution with (D + L)^T -- each by the oracle's own substitutions;
* ``ic0``          the zero-fill incomplete Cholesky factor: the lower-triangular
  C with the pattern of A's lower triangle whose product C C^T equals A on
  that pattern, row by row in the textbook (up-looking) order;
* ``ic0_apply``    z = (C C^T)^{-1} r: forward substitution with C, backward
  substitution with C^T;
* ``pcg``          preconditioned conjugate gradients (Hestenes-Stiefel form):
  r0 = b - A x0, z0 = M^{-1} r0, p0 = z0; per step alpha = (r, z) / (p, A p),
  x += alpha p, r -= alpha A p, stop when |r|_2 <= rtol |b|_2, z = M^{-1} r,
  beta = (r_new, z_new) / (r, z), p = z + beta p.

Parity status: pinned by tests against a dense solve, the dense M^{-1}, and
CG's property of reaching the solution of an n-dimensional system in at most
n steps (up to rounding) on small matrices; ic0 by numpy's Cholesky factor
where no fill arises (tridiagonal and dense patterns), by its defining
property C C^T = A on the pattern, and by one-step PCG convergence when the
factor is exact.
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


def ic0(Lo):
    """The IC(0) factor C of the SPD matrix whose lower triangle is Lo (same
    pattern, values replaced).  Row i, columns j < i ascending:
    C_ij = (A_ij - sum_{k < j} C_ik C_jk) / C_jj over the k stored in both
    rows, then C_ii = sqrt(A_ii - sum_{k < i} C_ik^2).  Raises on a
    non-positive pivot (the incomplete factorisation breaks down)."""
    n = Lo.n
    vals = Lo.val.astype(np.float64).copy()
    rows = []                                  # row i of C as {column: value}
    for i in range(n):
        a, e = int(Lo.row_ptr[i]), int(Lo.row_ptr[i + 1])
        ci = {}
        for p in range(a, e):
            j = int(Lo.col[p])
            s = float(Lo.val[p])
            if j < i:
                cj = rows[j]
                for k, v in ci.items():        # k < j: the entries already computed
                    if k in cj:
                        s -= v * cj[k]
                ci[j] = s / cj[j]
            else:
                s -= sum(v * v for k, v in ci.items())
                if not s > 0:
                    raise ValueError(f"IC(0) breaks down at row {i}: pivot {s}")
                ci[i] = float(np.sqrt(s))
            vals[p] = ci[j]
        rows.append(ci)
    return type(Lo)(n, Lo.row_ptr.copy(), Lo.col.copy(), vals)


def ic0_apply(C, r: np.ndarray) -> np.ndarray:
    """z = (C C^T)^{-1} r."""
    return backward_subst(transpose(C), forward_subst(C, r))


def pcg(A, b: np.ndarray, x0: np.ndarray, rtol: float, max_iter: int,
        precond: str = "sgs"):
    """(x, iterations, |r|_2 / |b|_2) of preconditioned CG with the symmetric
    Gauss-Seidel preconditioner built from A's lower triangle (``"sgs"``) or
    the IC(0) factor of A (``"ic0"``)."""
    Lo = lower_triangle(A)
    if precond == "ic0":
        C = ic0(Lo)

        def apply(r):
            return ic0_apply(C, r)
    elif precond == "sgs":
        def apply(r):
            return sgs_apply(Lo, r)
    else:
        raise ValueError(f"unknown preconditioner {precond!r}")
    x = np.array(x0, dtype=np.float64)
    r = b - _spmv(A, x)
    bnorm = float(np.sqrt(np.dot(b, b)))
    z = apply(r)
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
        z = apply(r)
        rz_new = float(np.dot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel

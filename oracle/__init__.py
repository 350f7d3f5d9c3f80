"""CPU oracle for the SpTRSV equation-rewriting path -- TEST INFRASTRUCTURE.

Only the tests under ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import or call anything
here.  The library itself (``paper_2103_11445_gb300``) never does, and this
package imports nothing from it: the two share no code.  The only common
dependency is ``matgen`` (seeded input generators, no method arithmetic).

Contents (each function cites the passage of the paper it follows):

* ``forward_subst``  serial FP64 CSR forward substitution (Sec. II, Fig. 1,
  Algorithm 1) -- C, ``sptrsv_oracle.c``;
* ``levels``         level of every row in DAG_L (Sec. II) -- C;
* ``residual``       r = b - L x -- C;
* ``backward_subst`` serial FP64 CSR backward substitution for an upper
  triangle (the mirror image of Algorithm 1) -- C;
* ``transpose``      CSR of A^T (scipy.sparse) and ``solve_op``: L x = b,
  U x = b, L^T x = b or U^T x = b by the substitution that operator needs;
* ``rewrite``        equation rewriting of one row (Sec. III, Figs. 2-3) and
  the thin-level selection heuristic -- Python, ``rewrite.py``;
* ``mlp``            FP64 forward/backward/Adam of the 3-layer cost-model
  network -- numpy, ``mlp.py``;
* ``pcg``            preconditioned conjugate gradients with the symmetric
  Gauss-Seidel preconditioner (two triangular solves per step) -- numpy and
  the substitutions above, ``pcg.py``;
* ``features``       per-level features of the matrix-analysis module (rows,
  entries, log2 row-length histogram, ancestor span, fill of each lift;
  Sec. IV) and the features of every candidate segment the per-segment cost
  network reads -- Python, ``features.py``;
* ``critpath``       weighted critical path of a (transformed) system and
  the critical-path-driven segment selection for synchronisation-free
  solves (Sec. III's remark that rewriting applies to them) -- Python,
  ``critpath.py``.

Parity status: every function above is pinned by tests against closed
forms, exact rational arithmetic, library routines or brute force; the
selection heuristic is the repository's own reading of the paper's manual
row choice (Sec. IV) and is pinned only by hand-worked examples.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sptrsv_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags, no -march, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or \
            os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            lib.oracle_forward_subst.argtypes = [ctypes.c_int32, i32p, i32p,
                                                 f64p, f64p, f64p,
                                                 ctypes.c_int32]
            lib.oracle_levels.argtypes = [ctypes.c_int32, i32p, i32p, i32p,
                                          ctypes.POINTER(ctypes.c_int32)]
            lib.oracle_spmv_lower.argtypes = [ctypes.c_int32, i32p, i32p, f64p,
                                              f64p, f64p, f64p, ctypes.c_int32]
            lib.oracle_backward_subst.argtypes = [ctypes.c_int32, i32p, i32p,
                                                  f64p, f64p, f64p,
                                                  ctypes.c_int32]
            for f in (lib.oracle_forward_subst, lib.oracle_levels,
                      lib.oracle_spmv_lower, lib.oracle_backward_subst):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


_ERR = {1: "column out of range or on the wrong side of the diagonal",
        2: "missing diagonal", 3: "zero diagonal"}

# which triangular operator a CSR stands for (same numbering as the library)
OP_LOWER, OP_UPPER, OP_LOWER_TRANS, OP_UPPER_TRANS = 0, 1, 2, 3


def _csr(A):
    return (np.ascontiguousarray(A.row_ptr, np.int32),
            np.ascontiguousarray(A.col, np.int32),
            np.ascontiguousarray(A.val, np.float64))


def forward_subst(A, b: np.ndarray) -> np.ndarray:
    """x = L^{-1} b by serial forward substitution (Sec. II, Algorithm 1).

    ``b`` is [n] or row-major [n, nrhs]; the result has the same shape."""
    rp, c, v = _csr(A)
    b2 = np.ascontiguousarray(b, np.float64).reshape(A.n, -1)
    x = np.empty_like(b2)
    rc = _load().oracle_forward_subst(A.n, rp, c, v, b2, x, b2.shape[1])
    if rc:
        raise ValueError(_ERR[rc])
    return x.reshape(np.shape(b))


def backward_subst(U, b: np.ndarray) -> np.ndarray:
    """x = U^{-1} b for an upper-triangular CSR by serial backward
    substitution (rows from last to first)."""
    rp, c, v = _csr(U)
    b2 = np.ascontiguousarray(b, np.float64).reshape(U.n, -1)
    x = np.empty_like(b2)
    rc = _load().oracle_backward_subst(U.n, rp, c, v, b2, x, b2.shape[1])
    if rc:
        raise ValueError(_ERR[rc])
    return x.reshape(np.shape(b))


def transpose(A):
    """CSR of A^T with ascending columns in every row (scipy.sparse)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).T.tocsr()
    M.sort_indices()
    return type(A)(A.n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                   M.data.astype(np.float64))


def solve_op(A, b: np.ndarray, op: int) -> np.ndarray:
    """Solution of op(A) x = b: A x for OP_LOWER / OP_UPPER, A^T x for the
    transposed operators, each by the substitution its triangle needs."""
    if op == OP_LOWER:
        return forward_subst(A, b)
    if op == OP_UPPER:
        return backward_subst(A, b)
    if op == OP_LOWER_TRANS:
        return backward_subst(transpose(A), b)
    if op == OP_UPPER_TRANS:
        return forward_subst(transpose(A), b)
    raise ValueError(f"unknown operator {op}")


def levels(A) -> tuple[np.ndarray, int]:
    """(level[n], number of levels) of DAG_L (Sec. II)."""
    rp, c, _ = _csr(A)
    lv = np.empty(A.n, np.int32)
    nl = ctypes.c_int32(0)
    rc = _load().oracle_levels(A.n, rp, c, lv, ctypes.byref(nl))
    if rc:
        raise ValueError(_ERR[rc])
    return lv, int(nl.value)


def level_sets(lv: np.ndarray, nlev: int) -> tuple[np.ndarray, np.ndarray]:
    """(level_ptr[nlev+1], perm[n]): rows grouped by level, ascending row
    index inside each level."""
    perm = np.argsort(lv, kind="stable").astype(np.int32)
    cnt = np.bincount(lv, minlength=nlev)
    ptr = np.zeros(nlev + 1, np.int64)
    np.cumsum(cnt, out=ptr[1:])
    return ptr.astype(np.int32), perm


def residual(A, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = b - L x."""
    rp, c, v = _csr(A)
    b2 = np.ascontiguousarray(b, np.float64).reshape(A.n, -1)
    x2 = np.ascontiguousarray(x, np.float64).reshape(A.n, -1)
    r = np.empty_like(b2)
    rc = _load().oracle_spmv_lower(A.n, rp, c, v, b2, x2, r, b2.shape[1])
    if rc:
        raise ValueError(_ERR[rc])
    return r.reshape(np.shape(b))


def relerr(x: np.ndarray, ref: np.ndarray) -> float:
    """max over right-hand sides of max_i |x_i - ref_i| / max_i |ref_i|."""
    x2 = np.asarray(x, np.float64).reshape(ref.shape[0], -1)
    r2 = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    num = np.abs(x2 - r2).max(axis=0)
    den = np.maximum(np.abs(r2).max(axis=0), np.finfo(np.float64).tiny)
    return float((num / den).max()) if r2.size else 0.0

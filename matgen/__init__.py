"""Seeded synthetic lower-triangular matrices and right-hand sides.

This module only builds inputs: CSR structure, values and right-hand sides
drawn from ``numpy.random.default_rng``.  It holds no step of the solver, of
the equation rewriting or of the cost model, and imports nothing else from
this repository, so both the CPU oracle and the CUDA library's tests can use
it without sharing any of the method's arithmetic.

Workloads (sizes and value distributions of the paper's setting, Section V,
which measures the SuiteSparse matrix lung2: a mostly serial matrix whose
levels are dominated by 2-row levels; that matrix is not available, so these
synthetic families stand in for it):

* ``stencil2d(64)``  lower triangle of the 2D 5-point Laplacian, natural
  ordering, diag 4, off-diagonal -1 (n = 4096, 127 levels);
* ``stencil3d(128)`` lower triangle of the 3D 7-point Laplacian, diag
  6 + U[0, 0.1], off-diagonal -1 (n = 2,097,152, 382 levels);
* ``thin_tail(1_000_000)`` 95% random-banded rows (8 distinct columns
  uniform in the 2000 rows above) then a 5% near-serial chain (row i-1 plus 3
  distinct random earlier rows); off-diagonal N(0,1)/(2*rowlen), diag
  1 + U[0, 1];
* ``batch(256)`` and ``costmodel_set(2000)`` mixtures of the three families.

Seeds follow ``config_index * 1000 + matrix_index``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "stencil2d", "stencil3d", "banded", "thin_tail", "chain",
    "random_lower", "batch_specs", "make_from_spec", "rhs_uniform",
    "manufactured_rhs", "config_matrix",
]


@dataclass
class CSR:
    """Lower-triangular matrix in CSR: columns ascending, diagonal last."""
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def _assemble(n: int, offs_lists: list[np.ndarray], masks: list[np.ndarray],
              offdiag_vals: list[np.ndarray], diag: np.ndarray) -> CSR:
    """Rows r carry entries at r - off for each (off, mask, value) triple.

    ``offs_lists`` must be given in descending offset order so that columns
    come out ascending; the diagonal is appended last."""
    rows = np.arange(n, dtype=np.int64)
    counts = np.ones(n, dtype=np.int64)
    for m in masks:
        counts += m
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    cursor = row_ptr[:-1].copy()
    for off, m, v in zip(offs_lists, masks, offdiag_vals):
        r = rows[m]
        col[cursor[m]] = (r - off).astype(np.int32)
        val[cursor[m]] = v[m] if np.ndim(v) else v
        cursor[m] += 1
    col[cursor] = rows.astype(np.int32)
    val[cursor] = diag
    return CSR(n, row_ptr.astype(np.int32), col, val)


def stencil2d(side: int, diag: float = 4.0) -> CSR:
    """Lower triangle of the 5-point Laplacian on a side x side grid.

    Row r = i*side + j holds (r - side, -1) if i > 0, (r - 1, -1) if j > 0
    and (r, diag)."""
    n = side * side
    r = np.arange(n)
    i, j = r // side, r % side
    return _assemble(n, [side, 1], [i > 0, j > 0], [-1.0, -1.0],
                     np.full(n, diag))


def stencil3d(side: int, seed: int = 1000, jitter: float = 0.1) -> CSR:
    """Lower triangle of the 7-point Laplacian on a side^3 grid.

    Row r = (i*side + j)*side + k holds -1 at r - side^2 (i > 0),
    r - side (j > 0), r - 1 (k > 0) and 6 + U[0, jitter] on the diagonal."""
    n = side ** 3
    rng = np.random.default_rng(seed)
    r = np.arange(n)
    i, j, k = r // (side * side), (r // side) % side, r % side
    diag = 6.0 + rng.uniform(0.0, jitter, n)
    return _assemble(n, [side * side, side, 1], [i > 0, j > 0, k > 0],
                     [-1.0, -1.0, -1.0], diag)


def _distinct_rows(rng: np.random.Generator, lo: np.ndarray, hi: np.ndarray,
                   k: int) -> np.ndarray:
    """k distinct integers uniform in [lo, hi) for every row (hi - lo > 4k).

    Rejection sampling: a row whose sorted draw holds a repeat is drawn
    again.  Returns int64 [rows, k], each row ascending."""
    out = np.empty((lo.size, k), dtype=np.int64)
    pending = np.arange(lo.size)
    width = hi - lo
    while pending.size:
        draw = lo[pending, None] + (rng.random((pending.size, k)) *
                                    width[pending, None]).astype(np.int64)
        draw.sort(axis=1)
        dup = (np.diff(draw, axis=1) == 0).any(axis=1)
        out[pending[~dup]] = draw[~dup]
        pending = pending[dup]
    return out


def _distinct_small(rng: np.random.Generator, lo: int, hi: int,
                    k: int) -> np.ndarray:
    w = hi - lo
    return np.sort(lo + rng.choice(w, size=min(k, w), replace=False))


def _from_flat(n: int, lens: np.ndarray, cols: np.ndarray, offdiag: np.ndarray,
               diag: np.ndarray) -> CSR:
    """CSR from row-ordered off-diagonal columns/values plus the diagonal."""
    lens = lens.astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens + 1, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = np.arange(cols.size, dtype=np.int64) + np.repeat(
        np.arange(n, dtype=np.int64), lens)
    col[pos] = cols
    val[pos] = offdiag
    dpos = row_ptr[1:] - 1
    col[dpos] = np.arange(n, dtype=np.int32)
    val[dpos] = diag
    return CSR(n, row_ptr.astype(np.int32), col, val)


def _from_row_lists(n: int, cols: list[np.ndarray], offdiag: list[np.ndarray],
                    diag: np.ndarray) -> CSR:
    lens = np.array([c.size for c in cols], dtype=np.int64)
    flat_c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    flat_v = np.concatenate(offdiag) if offdiag else np.zeros(0)
    return _from_flat(n, lens, flat_c, flat_v, diag)


def thin_tail(n: int = 1_000_000, seed: int = 2000, band: int = 2000,
              per_row: int = 8, chain_frac: float = 0.05,
              chain_extra: int = 3) -> CSR:
    """Random-banded head (per_row distinct columns uniform in
    [max(0, i-band), i-1]) and a near-serial chain tail (row i-1 plus
    chain_extra distinct columns uniform in [0, i-2]).

    Off-diagonal values N(0,1)/(2*rowlen), diagonal 1 + U[0,1]."""
    rng = np.random.default_rng(seed)
    n_chain = int(round(n * chain_frac))
    n_band = n - n_chain
    pieces: list[np.ndarray] = []
    lens = np.zeros(n, dtype=np.int64)
    # banded head: narrow windows near the top exactly, the rest vectorised
    cut = min(n_band, 4 * per_row + 1)
    for i in range(cut):
        c = _distinct_small(rng, max(0, i - band), i, per_row)
        pieces.append(c)
        lens[i] = c.size
    if n_band > cut:
        rows = np.arange(cut, n_band, dtype=np.int64)
        lo = np.maximum(rows - band, 0)
        blk = _distinct_rows(rng, lo, rows, per_row)
        pieces.append(blk.ravel())
        lens[cut:n_band] = per_row
    # chain tail
    for i in range(n_band, min(n, n_band + 4 * chain_extra + 2)):
        extra = (_distinct_small(rng, 0, i - 1, chain_extra) if i >= 2
                 else np.zeros(0, np.int64))
        c = np.concatenate([extra, [i - 1]]) if i >= 1 else extra
        pieces.append(c.astype(np.int64))
        lens[i] = c.size
    start = n_band + 4 * chain_extra + 2
    if n > start:
        rows = np.arange(start, n, dtype=np.int64)
        extra = _distinct_rows(rng, np.zeros_like(rows), rows - 1, chain_extra)
        blk = np.concatenate([extra, (rows - 1)[:, None]], axis=1)
        pieces.append(blk.ravel())
        lens[start:] = chain_extra + 1
    cols = np.concatenate(pieces) if pieces else np.zeros(0, np.int64)
    rowlen = np.repeat(lens, lens)
    vals = rng.standard_normal(cols.size) / (2.0 * np.maximum(rowlen, 1))
    diag = 1.0 + rng.uniform(0.0, 1.0, n)
    return _from_flat(n, lens, cols, vals, diag)


def banded(n: int, seed: int, band: int = 2000, per_row: int = 8) -> CSR:
    """Random-banded rows only (the head of ``thin_tail``)."""
    return thin_tail(n, seed=seed, band=band, per_row=per_row, chain_frac=0.0)


def chain(n: int, a: float = 1.0, diag: float = 1.0) -> CSR:
    """Bidiagonal chain: diag on the diagonal, -a below it."""
    r = np.arange(n)
    return _assemble(n, [1], [r > 0], [-a], np.full(n, diag))


def random_lower(n: int, seed: int, density: float = 0.3,
                 integer: bool = False, diag_min: float = 1.0) -> CSR:
    """Small dense-ish random lower-triangular matrix (test sizes only).

    ``integer`` draws off-diagonal entries from {-3..3} \\ {0} and diagonals
    from {1..4} so that exact rational arithmetic stays small."""
    rng = np.random.default_rng(seed)
    cols, vals = [], []
    for i in range(n):
        m = rng.random(i) < density
        c = np.nonzero(m)[0].astype(np.int64)
        if integer:
            v = rng.integers(1, 4, c.size) * rng.choice([-1, 1], c.size)
            v = v.astype(np.float64)
        else:
            v = rng.standard_normal(c.size) / max(1, c.size)
        cols.append(c)
        vals.append(v)
    if integer:
        diag = rng.integers(1, 5, n).astype(np.float64)
    else:
        diag = diag_min + rng.random(n)
    return _from_row_lists(n, cols, vals, diag)


def transposed(A: CSR) -> CSR:
    """The same entries stored as A^T (a lower matrix becomes an upper one):
    entries ordered by (column, row) with a stable sort, CSR of the result
    (an input rearrangement, no arithmetic on the values)."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.row_ptr))
    order = np.lexsort((rows, A.col))
    cnt = np.bincount(A.col, minlength=A.n)
    ptr = np.zeros(A.n + 1, np.int64)
    np.cumsum(cnt, out=ptr[1:])
    return CSR(A.n, ptr.astype(np.int32), rows[order].astype(np.int32),
               np.ascontiguousarray(A.val[order]))


def symmetric_from_lower(L: CSR) -> CSR:
    """The symmetric matrix whose lower triangle (diagonal included) is L:
    L's entries plus the mirror image of its off-diagonal ones, CSR with
    ascending columns (an input rearrangement, no arithmetic on values)."""
    rows = np.repeat(np.arange(L.n, dtype=np.int64), np.diff(L.row_ptr))
    off = L.col != rows
    r = np.concatenate([rows, L.col[off].astype(np.int64)])
    c = np.concatenate([L.col.astype(np.int64), rows[off]])
    v = np.concatenate([L.val, L.val[off]])
    order = np.lexsort((c, r))
    cnt = np.bincount(r, minlength=L.n)
    ptr = np.zeros(L.n + 1, np.int64)
    np.cumsum(cnt, out=ptr[1:])
    return CSR(L.n, ptr.astype(np.int32), c[order].astype(np.int32),
               np.ascontiguousarray(v[order]))


def rhs_uniform(n: int, nrhs: int = 1, seed: int = 7) -> np.ndarray:
    """b ~ U[-1, 1], row-major [n, nrhs] (shape [n] when nrhs == 1)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, (n, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b


def manufactured_rhs(A: CSR, x_true: np.ndarray) -> np.ndarray:
    """b = L x_true (input construction for manufactured-solution cases)."""
    x2 = x_true.reshape(A.n, -1)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    b = np.zeros_like(x2)
    np.add.at(b, rows, A.val[:, None] * x2[A.col])
    return b.reshape(x_true.shape)


# --- mixtures -------------------------------------------------------------

def batch_specs(count: int = 256, seed: int = 4000, n_lo: float = 1e3,
                n_hi: float = 2e5, nrhs_max: int = 32,
                band_range: tuple[int, int] = (8, 8)) -> list[dict]:
    """Specs of a mixture: n log-uniform in [n_lo, n_hi], family uniform in
    {5-point, 7-point, random-banded}, nrhs uniform in {1..nrhs_max}.

    Stencil grids take side round(sqrt(n)) or round(cbrt(n)), so n is
    adjusted to the grid."""
    rng = np.random.default_rng(seed)
    specs = []
    for m in range(count):
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        fam = ("stencil2d", "stencil3d", "banded")[int(rng.integers(0, 3))]
        nrhs = int(rng.integers(1, nrhs_max + 1))
        per_row = int(rng.integers(band_range[0], band_range[1] + 1))
        if fam == "stencil2d":
            side = max(2, int(round(n ** 0.5)))
            n_adj = side * side
        elif fam == "stencil3d":
            side = max(2, int(round(n ** (1.0 / 3.0))))
            n_adj = side ** 3
        else:
            side = 0
            n_adj = int(round(n))
        specs.append(dict(index=m, family=fam, n=n_adj, side=side, nrhs=nrhs,
                          per_row=per_row, seed=seed + m))
    return specs


def make_from_spec(spec: dict) -> CSR:
    fam = spec["family"]
    if fam == "stencil2d":
        return stencil2d(spec["side"])
    if fam == "stencil3d":
        return stencil3d(spec["side"], seed=spec["seed"])
    if fam == "banded":
        return banded(spec["n"], seed=spec["seed"],
                      per_row=spec.get("per_row", 8))
    if fam == "thin_tail":
        return thin_tail(spec["n"], seed=spec["seed"], per_row=spec.get("per_row", 8),
                         chain_frac=spec.get("chain_frac", 0.05))
    raise ValueError(f"unknown family {fam}")


def costmodel_specs(count: int = 2000, seed: int = 5000) -> list[dict]:
    """The cost-model mixture: n log-uniform in [1e4, 5e5], families as in
    ``batch_specs``, random-banded rows with 5..20 off-diagonal entries."""
    return batch_specs(count, seed=seed, n_lo=1e4, n_hi=5e5, nrhs_max=1,
                       band_range=(5, 20))


def costmodel_large_specs(count: int = 80, seed: int = 7000) -> list[dict]:
    """Larger matrices for the cost model's training set only: n log-uniform
    in [5e5, 2.5e6], family uniform in {5-point, 7-point, random-banded,
    thin-tail} (thin tails with a chain of 1-10 % of the rows)."""
    rng = np.random.default_rng(seed)
    specs = []
    for m in range(count):
        n = float(np.exp(rng.uniform(np.log(5e5), np.log(2.5e6))))
        fam = ("stencil2d", "stencil3d", "banded", "thin_tail")[int(rng.integers(0, 4))]
        per_row = int(rng.integers(5, 13))
        if fam == "stencil2d":
            side = int(round(n ** 0.5))
            n_adj = side * side
        elif fam == "stencil3d":
            side = int(round(n ** (1.0 / 3.0)))
            n_adj = side ** 3
        else:
            side = 0
            n_adj = int(round(n))
        specs.append(dict(index=m, family=fam, n=n_adj, side=side, nrhs=1, per_row=per_row,
                          chain_frac=float(rng.uniform(0.01, 0.10)), seed=seed + m))
    return specs


def segmodel_specs(count: int = 40, seed: int = 8000) -> list[dict]:
    """Matrices of the per-segment cost network's data: n log-uniform in
    [3e4, 2e5], family uniform in {5-point, 7-point, random-banded,
    thin-tail} (random-banded rows with 5..12 entries, thin tails with a
    chain of 1-10 % of the rows)."""
    rng = np.random.default_rng(seed)
    specs = []
    for m in range(count):
        n = float(np.exp(rng.uniform(np.log(3e4), np.log(2e5))))
        fam = ("stencil2d", "stencil3d", "banded", "thin_tail")[int(rng.integers(0, 4))]
        per_row = int(rng.integers(5, 13))
        if fam == "stencil2d":
            side = int(round(n ** 0.5))
            n_adj = side * side
        elif fam == "stencil3d":
            side = int(round(n ** (1.0 / 3.0)))
            n_adj = side ** 3
        else:
            side = 0
            n_adj = int(round(n))
        specs.append(dict(index=m, family=fam, n=n_adj, side=side, nrhs=1, per_row=per_row,
                          chain_frac=float(rng.uniform(0.01, 0.10)), seed=seed + m))
    return specs


def segmodel_large_specs() -> list[dict]:
    """Large training-only matrices of the per-segment network: 7-point
    stencils of side 90, 110 and 120 (not the benchmark's 128),
    5-point of side 800 and 1200, thin tails of 5e5 and 1e6 rows, a
    random-banded matrix of 6e5 rows."""
    specs = []
    for k, (fam, size) in enumerate((("stencil3d", 90), ("stencil3d", 110), ("stencil3d", 120),
                                     ("stencil2d", 800), ("stencil2d", 1200),
                                     ("thin_tail", 500_000), ("thin_tail", 1_000_000),
                                     ("banded", 600_000))):
        side = size if fam.startswith("stencil") else 0
        n = side ** 3 if fam == "stencil3d" else side ** 2 if fam == "stencil2d" else size
        specs.append(dict(index=k, family=fam, n=n, side=side, nrhs=1, per_row=8,
                          chain_frac=0.05, seed=8500 + k))
    return specs


def config_matrix(index: int, small: bool = False) -> CSR:
    """The matrix of workload ``index`` (1-based as listed in the module doc).

    ``small`` gives a shrunken copy of the same family for fast tests."""
    if index == 1:
        return stencil2d(16 if small else 64)
    if index == 2:
        return stencil3d(16 if small else 128, seed=2 * 1000)
    if index == 3:
        return thin_tail(20_000 if small else 1_000_000, seed=3 * 1000)
    raise ValueError("workloads 4 and 5 are mixtures: use batch_specs")

"""Oracle for the per-level features of the matrix-analysis module --
TEST INFRASTRUCTURE (only tests, the smoke check and the benchmark's CPU
legs use it).

The paper's matrix-analysis module (Sec. IV) inspects the levels before the
rewriting chooses rows; the features here are what a row choice per level
needs (the definitions are this repository's reading):

per level l (rows i with level(i) = l), in this order:
  0  rows
  1  off-diagonal entries of its rows (nnz of the level)
  2..9  row-length histogram, 8 log2 bins of the off-diagonal count c:
        bin 0: c = 0; bin b (1..6): 2^(b-1) <= c < 2^b; bin 7: c >= 64
  10 ancestor span: the most levels between a row of l and the lowest level
     it depends on, max over rows of (l - min level of its dependencies),
     0 for rows without dependencies
  11.. for r = 1..lifts: FLOPs added when every row of l is lifted to
     target level l - r (rewritten to depend only on levels < l - r,
     Sec. III), 2 per added off-diagonal term (x or b), summed over the
     level; -1 when a row would exceed the fill cap; 0 when l < r.
"""
from __future__ import annotations

import numpy as np

from .rewrite import _row, rewrite_row

N_BASE = 11


def length_bin(c: int) -> int:
    if c <= 0:
        return 0
    b = int(c).bit_length()          # 2^(b-1) <= c < 2^b
    return min(b, 7)


def level_features(A, level: np.ndarray, nlev: int, lifts: int, cap: int) -> np.ndarray:
    F = N_BASE + lifts
    out = np.zeros((nlev, F), dtype=np.float64)
    by_level: list[list[int]] = [[] for _ in range(nlev)]
    for i in range(A.n):
        by_level[int(level[i])].append(i)
    for lv in range(nlev):
        span = 0
        for i in by_level[lv]:
            cols, _, _ = _row(A, i)
            c = int(cols.size)
            out[lv, 0] += 1
            out[lv, 1] += c
            out[lv, 2 + length_bin(c)] += 1
            if c:
                span = max(span, lv - int(min(level[j] for j in cols.tolist())))
        out[lv, 10] = span
        for r in range(1, lifts + 1):
            if lv < r:
                continue
            tot = 0
            for i in by_level[lv]:
                rw = rewrite_row(A, level, i, lv - r)
                if rw.fill > cap:
                    tot = -1
                    break
                tot += 2 * (rw.fill - int(_row(A, i)[0].size))
            out[lv, N_BASE + r - 1] = tot
    return out


N_SEG = 8


def segment_features(A, level: np.ndarray, nlev: int, d_max: int, cap: int):
    """Features of every candidate segment (kept level t, depth d: levels
    t..t+d merged, the rows of t+1..t+d rewritten to depend on levels < t),
    the inputs of the per-segment cost network (this repository's reading,
    Sec. IV):
      0 log2(1 + rows), 1 log2(1 + x and b terms), 2 log2(1 + most terms of a
      row), 3 terms per row, 4 d, 5 fraction of rows rewritten, 6 log2 n,
      7 log2(nnz / n) (nnz with the diagonal).
    terms = the kept level's off-diagonal entries plus, per lifted level,
    its entries and the terms its lift adds; the most terms of a row come
    from the lift table.  ok[t, d] = False where t + d runs past the last
    level or a lifted row exceeds the fill cap (and for every deeper d)."""
    from .critpath import lift_table
    base = level_features(A, level, nlev, d_max, cap)
    table = lift_table(A, level, nlev, d_max, cap)
    nnz = int(A.row_ptr[-1])
    feat = np.zeros((nlev, d_max + 1, N_SEG))
    ok = np.zeros((nlev, d_max + 1), dtype=bool)
    for t in range(nlev):
        rows = terms = rew = 0.0
        maxt = 0.0
        for d in range(d_max + 1):
            lv = t + d
            if lv >= nlev:
                break
            if d == 0:
                terms += base[lv, 1]
                maxt = table[(lv, 0)]
            else:
                added = base[lv, N_BASE + d - 1]
                if added < 0 or table.get((lv, d)) is None:
                    break
                terms += base[lv, 1] + added / 2.0
                maxt = max(maxt, table[(lv, d)])
                rew += base[lv, 0]
            rows += base[lv, 0]
            feat[t, d] = (np.log2(1 + rows), np.log2(1 + terms), np.log2(1 + maxt),
                          terms / max(rows, 1.0), d, rew / max(rows, 1.0),
                          np.log2(max(A.n, 1)), np.log2(max(nnz, 1) / max(A.n, 1)))
            ok[t, d] = True
    return feat, ok

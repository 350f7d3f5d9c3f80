"""Oracle for the equation-rewriting transformation -- TEST INFRASTRUCTURE.

Only tests, the smoke check and the benchmark's CPU legs use this module.

Sec. III of the paper rewrites the equation of a row by substituting the
equation of one of its dependencies: the dependency edge disappears, the
dependency's own dependencies become the row's, and the row moves up one
level (Fig. 2, where row 3 is rewritten first with row 1's original equation
and then with row 0's).  Repeating this until the row only depends on rows of
levels below a target level t lifts the row into level t.  Rearranged back
into L x = b form (Fig. 3) the row keeps its diagonal, gets new coefficients
on the unknowns it still depends on, and a right-hand side in which other
entries of b appear with weights.

Readings taken here (the figures holding the worked example are not
available):
* a step substitutes the *original* equation of the dependency (Fig. 2's
  caption), always the highest-numbered dependency that is still at level
  >= t; any order gives the same rearranged row, because the result is the
  unique combination  row_i - sum_{j in S} c_j row_j  that cancels every
  column of S (S = the dependencies eliminated);
* explicit zeros produced by cancellation stay as stored entries (the
  pattern is structural, as is DAG_L);
* the updated right-hand side is kept symbolic:  b'_i = b_i - sum c_j b_j,
  evaluated at solve time because b is an input of every solve;
* repeated unknowns after substitution are merged into one term (the
  grouping Sec. IV lists as a planned optimisation).

FLOPs of a row (used by the selection heuristic): 2 per off-diagonal term,
x-part and b-part alike, plus 1 for the diagonal.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field

import numpy as np


@dataclass
class RewrittenRow:
    """x_i = (b_i - sum_j bw[j] * b[bcol[j]] - sum_k xv[k] * x[xcol[k]]) / diag."""
    row: int
    target: int
    xcol: np.ndarray   # int32, ascending, every column at level < target
    xval: np.ndarray   # float64
    bcol: np.ndarray   # int32, ascending: the eliminated dependencies S
    bw: np.ndarray     # float64
    diag: float

    @property
    def fill(self) -> int:
        return int(self.xcol.size + self.bcol.size)


def _row(A, i):
    a, e = int(A.row_ptr[i]), int(A.row_ptr[i + 1])
    # the diagonal is the last stored entry of a sorted lower-triangular row
    return A.col[a:e - 1], A.val[a:e - 1], float(A.val[e - 1])


def rewrite_row(A, level: np.ndarray, i: int, t: int) -> RewrittenRow:
    """Rewrite row i until it depends only on rows of level < t (Sec. III).

    Each step takes the largest dependency j with level[j] >= t, solves row
    j's original equation for x_j and substitutes it into row i:
        m = coef_i[j] / L[j][j];  coef_i[k] -= m * L[j][k]  (k < j);
        coef_i[j] = 0;  c_j += m   (b'_i = b_i - sum c_j b_j).
    New dependencies are always below j, so each j is substituted once."""
    cols, vals, d = _row(A, i)
    coef: dict[int, float] = {}
    for k, v in zip(cols.tolist(), vals.tolist()):
        coef[k] = v
    heap = [-k for k in coef if level[k] >= t]
    heapq.heapify(heap)
    c: dict[int, float] = {}
    while heap:
        j = -heapq.heappop(heap)
        jc, jv, jd = _row(A, j)
        m = coef.pop(j) / jd
        c[j] = m
        for k, v in zip(jc.tolist(), jv.tolist()):
            if k not in coef:
                coef[k] = 0.0
                if level[k] >= t:
                    heapq.heappush(heap, -k)
            coef[k] -= m * v
    xc = np.array(sorted(coef), dtype=np.int32)
    xv = np.array([coef[k] for k in xc.tolist()], dtype=np.float64)
    bc = np.array(sorted(c), dtype=np.int32)
    bw = np.array([c[k] for k in bc.tolist()], dtype=np.float64)
    return RewrittenRow(i, t, xc, xv, bc, bw, d)


def rewritten_fill(A, level: np.ndarray, i: int, t: int) -> int:
    """Number of off-diagonal terms (x-part + b-part) of row i lifted to t."""
    return rewrite_row(A, level, i, t).fill


def offdiag_counts(A) -> np.ndarray:
    return (np.diff(A.row_ptr) - 1).astype(np.int64)


def total_flops(A) -> int:
    """2 per off-diagonal term plus 1 per row (one right-hand side)."""
    return int(2 * offdiag_counts(A).sum() + A.n)


def select_segments(level_rows: np.ndarray, added, tau: int, d_max: int,
                    rho: float, base_flops: int) -> list[tuple[int, int]]:
    """Thin-level merging heuristic H: the repository's reading of the row
    choice the paper leaves to the programmer (Sec. IV) and of its
    experiment (Sec. V: thin levels removed, +10% FLOPs).

    Levels are scanned in order.  Each segment starts at a kept level t; the
    following levels t+1, t+2, ... are merged into it (their rows rewritten to
    target t) while
      * the level has fewer than ``tau`` rows (it is thin),
      * fewer than ``d_max`` levels have been merged into this segment,
      * the rewrite fits (``added(l, r)`` is not None: no row exceeds the
        fill cap), and
      * the FLOPs added over the whole matrix stay <= rho * base_flops.
    ``added(l, r)`` = FLOPs added by rewriting every row of level l to
    target l - r.  Returns [(t, d)]: levels t..t+d form one new level."""
    nlev = len(level_rows)
    budget = rho * float(base_flops)
    used = 0
    segs: list[tuple[int, int]] = []
    lv = 0
    while lv < nlev:
        t, d = lv, 0
        while d < d_max and t + d + 1 < nlev and level_rows[t + d + 1] < tau:
            cost = added(t + d + 1, d + 1)
            if cost is None or float(used + cost) > budget:
                break
            used += cost
            d += 1
        segs.append((t, d))
        lv = t + d + 1
    return segs


@dataclass
class Transformed:
    """Result of the oracle transformation."""
    level: np.ndarray            # original level of each row
    nlev: int
    segments: list               # [(t, d)]
    new_level: np.ndarray        # new level (segment index) of each row
    rows: dict = field(default_factory=dict)  # row -> RewrittenRow (rewritten rows only)
    added_flops: int = 0

    @property
    def nlev_new(self) -> int:
        return len(self.segments)


def transform(A, level: np.ndarray, nlev: int, tau: int, d_max: int,
              rho: float, max_fill: int) -> Transformed:
    """Full oracle transformation: candidate fills, heuristic H, rewrite."""
    offd = offdiag_counts(A)
    by_level: list[list[int]] = [[] for _ in range(nlev)]
    for r in range(A.n):
        by_level[int(level[r])].append(r)
    level_rows = np.array([len(x) for x in by_level], dtype=np.int64)
    cache: dict = {}

    def added(lv: int, r: int):
        key = (lv, r)
        if key not in cache:
            tot = 0
            for i in by_level[lv]:
                f = rewritten_fill(A, level, i, lv - r)
                if f > max_fill:
                    cache[key] = None
                    break
                tot += 2 * (f - int(offd[i]))
            else:
                cache[key] = tot
        return cache[key]

    segs = select_segments(level_rows, added, tau, d_max, rho, total_flops(A))
    new_level = np.empty(A.n, dtype=np.int32)
    out = Transformed(level, nlev, segs, new_level)
    for s, (t, d) in enumerate(segs):
        for lv in range(t, t + d + 1):
            for i in by_level[lv]:
                new_level[i] = s
                if lv > t:
                    rw = rewrite_row(A, level, i, t)
                    out.rows[i] = rw
                    out.added_flops += 2 * (rw.fill - int(offd[i]))
    return out


def solve_transformed(A, tr: Transformed, b: np.ndarray) -> np.ndarray:
    """Serial solve of the transformed system, new level by new level.

    Asserts the schedule is valid: every x term of a row refers to a row of
    an earlier new level."""
    b2 = np.asarray(b, np.float64).reshape(A.n, -1)
    x = np.full_like(b2, np.nan)
    done = np.zeros(A.n, dtype=bool)
    order = np.lexsort((np.arange(A.n), tr.new_level))
    for i in order.tolist():
        if i in tr.rows:
            rw = tr.rows[i]
            xc, xv, bc, bw, d = rw.xcol, rw.xval, rw.bcol, rw.bw, rw.diag
        else:
            xc, xv, d = _row(A, i)
            bc, bw = np.zeros(0, np.int32), np.zeros(0)
        assert all(tr.new_level[k] < tr.new_level[i] for k in xc.tolist())
        s = b2[i].copy()
        for j, w in zip(bc.tolist(), bw.tolist()):
            s -= w * b2[j]
        for k, v in zip(xc.tolist(), xv.tolist()):
            assert done[k]
            s -= v * x[k]
        x[i] = s / d
        done[i] = True
    return x.reshape(np.shape(b))

"""Oracle for the critical-path-driven rewrite selection -- TEST INFRASTRUCTURE.

Only tests, the smoke check and the benchmark's CPU legs use this module.

The paper notes that the rewriting applies to synchronisation-free execution
as well as to level sets (Sec. III), and leaves the choice of rows to the
programmer (Sec. IV).  A synchronisation-free solve has no barriers: a row
can finish only after the latest of its dependencies has finished, and then
it still pays one hop (the dependency's value reaching it) and its own
terms.  The readings taken here:

* weighted critical path of a (transformed) lower-triangular system:
      f(i) = H + t(i) + max_{j in deps(i)} f(j)      (max over nothing = 0),
      CP   = max_i f(i),
  with t(i) the row's off-diagonal terms (x terms, plus the b terms of a
  rewritten row: every one is a multiply-add on the row's path) and deps(i)
  the unknowns its x terms read; H is the hop weight in units of one term;
* level-set model of a segmentation: a segment (t, d) merges levels
  t..t+d into one new level (the rows of t+1..t+d rewritten to depend on
  levels < t only).  If every row of a new level waits for the whole level
  before it, the plan's critical path is
      CP_lev = sum over new levels of (H + max terms of a row in it),
  an upper bound of the true CP of the transformed system (each row's f is
  at most the sum over the new levels up to its own);
* the selection (SELECT_CRITPATH) minimises CP_lev over all segmentations
  with at most d_max levels absorbed per segment and no rewritten row above
  the fill cap, by dynamic programming from the last level down; ties go to
  the smaller d (fewer rewritten rows).

Pinned by tests/test_oracle_critpath.py: closed forms on chains, a hand-worked
DAG, networkx's longest path on random DAGs, brute force over all
segmentations of small matrices, and the upper-bound property on rewritten
systems built by oracle.rewrite.
"""
from __future__ import annotations

import numpy as np

from .rewrite import _row, rewrite_row


def critical_path(deps: list, terms: list, H: int) -> tuple[int, np.ndarray]:
    """CP and f(i) for rows given in an order where every dependency comes
    first (deps[i]: iterable of row indices < i, terms[i]: the row's
    off-diagonal term count)."""
    n = len(deps)
    f = np.zeros(n, dtype=np.int64)
    for i in range(n):
        m = 0
        for j in deps[i]:
            assert j < i
            m = max(m, int(f[j]))
        f[i] = H + int(terms[i]) + m
    return (int(f.max()) if n else 0), f


def plain_rows(A):
    """deps and terms of the plain system (its rows as stored)."""
    deps, terms = [], []
    for i in range(A.n):
        cols, _, _ = _row(A, i)
        deps.append(cols.tolist())
        terms.append(int(cols.size))
    return deps, terms


def transformed_rows(A, level: np.ndarray, segments) -> tuple[list, list]:
    """deps and terms of the system the segmentation gives (rows of absorbed
    levels rewritten to their segment's kept level with oracle.rewrite)."""
    deps, terms = plain_rows(A)
    tgt = {}
    for (t, d) in segments:
        for lv in range(t + 1, t + d + 1):
            tgt[lv] = t
    for i in range(A.n):
        lv = int(level[i])
        if lv in tgt:
            rw = rewrite_row(A, level, i, tgt[lv])
            deps[i] = rw.xcol.tolist()
            terms[i] = rw.fill
    return deps, terms


def levelset_cp(max_terms_of_new_levels, H: int) -> int:
    """CP_lev: sum over new levels of H + (max terms of a row in it)."""
    return int(sum(H + int(m) for m in max_terms_of_new_levels))


def lift_table(A, level: np.ndarray, nlev: int, d_max: int, cap: int) -> dict:
    """maxterms[(l, r)]: the most off-diagonal terms of a row of level l
    rewritten to level l - r (r = 0: as stored); None if some row of the
    level would exceed the fill cap."""
    by_level: list[list[int]] = [[] for _ in range(nlev)]
    for i in range(A.n):
        by_level[int(level[i])].append(i)
    table = {}
    for lv in range(nlev):
        table[(lv, 0)] = max((int(_row(A, i)[0].size) for i in by_level[lv]), default=0)
        for r in range(1, min(d_max, lv) + 1):
            m = 0
            for i in by_level[lv]:
                f = rewrite_row(A, level, i, lv - r).fill
                if f > cap:
                    m = None
                    break
                m = max(m, f)
            table[(lv, r)] = m
    return table


def select_critpath(nlev: int, table: dict, H: int, d_max: int) -> list[tuple[int, int]]:
    """The segmentation minimising CP_lev (dynamic programming over the kept
    levels, last level first): best[t] = min over feasible d of
        H + max(table[(t, 0)], table[(t + r, r)] for r = 1..d) + best[t + d + 1]."""
    INF = float("inf")
    best = [INF] * (nlev + 1)
    choice = [0] * (nlev + 1)
    best[nlev] = 0
    for t in range(nlev - 1, -1, -1):
        m = table[(t, 0)]
        for d in range(0, d_max + 1):
            if t + d >= nlev:
                break
            if d > 0:
                v = table.get((t + d, d))
                if v is None:
                    break           # deeper merges of this segment lift this level too
                m = max(m, v)
            c = H + m + best[t + d + 1]
            if c < best[t]:
                best[t], choice[t] = c, d
    segs, t = [], 0
    while t < nlev:
        segs.append((t, choice[t]))
        t += choice[t] + 1
    return segs


def segments_cp(segments, table: dict, H: int) -> int:
    """CP_lev of a segmentation from the lift table."""
    tot = 0
    for (t, d) in segments:
        m = table[(t, 0)]
        for r in range(1, d + 1):
            m = max(m, table[(t + r, r)])
        tot += H + m
    return tot


def select_min_sum(cost: np.ndarray, ok: np.ndarray) -> list[tuple[int, int]]:
    """The segmentation minimising the sum of per-segment costs (the
    per-segment learned cost of SELECT_SEGMODEL): cost[t, d] the cost of the
    segment merging levels t..t+d, ok[t, d] whether it exists.  Dynamic
    programming from the last level down, best[t] = min over d of
    cost[t, d] + best[t + d + 1], a depth stopping at its first missing
    segment, ties to the smaller d."""
    nlev, D = cost.shape
    best = [float("inf")] * (nlev + 1)
    choice = [0] * (nlev + 1)
    best[nlev] = 0.0
    for t in range(nlev - 1, -1, -1):
        for d in range(D):
            if t + d >= nlev or not ok[t, d]:
                break
            c = float(cost[t, d]) + best[t + d + 1]
            if c < best[t]:
                best[t], choice[t] = c, d
    segs, t = [], 0
    while t < nlev:
        segs.append((t, choice[t]))
        t += choice[t] + 1
    return segs

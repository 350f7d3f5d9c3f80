"""Pins of the rewriting oracle (Sec. III, Figs. 2-3) against closed forms,
the dense elimination formula c^T = L[i,S] L[S,S]^{-1} computed by numpy and
by exact rational arithmetic, and the invariants of the transformed system;
plus hand-worked runs of the thin-level selection heuristic."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import matgen as mg
import oracle
from oracle import rewrite as rw


def dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def eliminated_set(A, level, i, t):
    """Dependencies reachable from row i through rows of level >= t (BFS,
    independent of the oracle's substitution loop)."""
    seen, stack = set(), [i]
    while stack:
        r = stack.pop()
        for k in range(A.row_ptr[r], A.row_ptr[r + 1] - 1):
            j = int(A.col[k])
            if level[j] >= t and j not in seen:
                seen.add(j)
                stack.append(j)
    return sorted(seen)


# --- closed forms -----------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 7])
def test_chain_closed_form(d):
    # x_i - a x_{i-1} = b_i; lifting row t+r to level t gives
    #   x_i - a^(r+1) x_{t-1} = b_i + sum_{k=1..r} a^k b_{i-k}
    m, a = 40, 0.5
    A = mg.chain(m, a=a, diag=1.0)
    lv, nl = oracle.levels(A)
    tr = rw.transform(A, lv, nl, tau=10**9, d_max=d, rho=float("inf"),
                      max_fill=10**9)
    assert tr.nlev_new == -(-m // (d + 1))
    for i, row in tr.rows.items():
        t = row.target
        r = i - t
        assert t % (d + 1) == 0 and 1 <= r <= d
        if t == 0:
            assert row.xcol.size == 0
        else:
            assert row.xcol.tolist() == [t - 1]
            assert row.xval[0] == -(a ** (r + 1))
        assert row.bcol.tolist() == list(range(t, i))
        assert row.bw.tolist() == [-(a ** (i - j)) for j in range(t, i)]
    b = mg.rhs_uniform(m, seed=1)
    assert oracle.relerr(rw.solve_transformed(A, tr, b),
                         oracle.forward_subst(A, b)) < 1e-15


def fig2_matrix():
    # rows 0..3: row 1 depends on row 0, row 2 on row 0, row 3 on row 1
    l00, l10, l11, l20, l22, l31, l33 = 2.0, 0.5, 4.0, -1.0, 8.0, 3.0, 0.25
    rp = np.array([0, 1, 3, 5, 7], np.int32)
    col = np.array([0, 0, 1, 0, 2, 1, 3], np.int32)
    val = np.array([l00, l10, l11, l20, l22, l31, l33])
    return mg.CSR(4, rp, col, val), (l00, l10, l11, l31, l33)


def test_fig2_two_substitutions():
    # row 3 -> rewritten with row 1, then with row 0: no dependency left,
    # x3 = (b3 - (l31/l11) b1 + (l31 l10 / (l11 l00)) b0) / l33
    A, (l00, l10, l11, l31, l33) = fig2_matrix()
    lv, nl = oracle.levels(A)
    assert lv.tolist() == [0, 1, 1, 2] and nl == 3
    row = rw.rewrite_row(A, lv, 3, 0)
    assert row.xcol.size == 0
    assert row.bcol.tolist() == [0, 1]
    c0, c1 = row.bw.tolist()
    assert Fraction(c1) == Fraction(l31) / Fraction(l11)
    assert Fraction(c0) == -Fraction(l31) * Fraction(l10) / (Fraction(l11) * Fraction(l00))
    assert row.diag == l33


def test_fig2_one_substitution():
    # one step: row 3 keeps a dependency on row 0 and moves up one level
    A, (l00, l10, l11, l31, l33) = fig2_matrix()
    lv, _ = oracle.levels(A)
    row = rw.rewrite_row(A, lv, 3, 1)
    assert row.xcol.tolist() == [0] and row.bcol.tolist() == [1]
    assert Fraction(row.xval[0]) == -Fraction(l31) * Fraction(l10) / Fraction(l11)
    assert Fraction(row.bw[0]) == Fraction(l31) / Fraction(l11)


# --- dense elimination formula -------------------------------------------------

def cases(seed, n=60, density=0.12, integer=False):
    A = mg.random_lower(n, seed=seed, density=density, integer=integer)
    lv, _ = oracle.levels(A)
    rng = np.random.default_rng(seed)
    rows = [i for i in range(n) if lv[i] >= 2]
    out = []
    for i in rng.choice(rows, size=min(8, len(rows)), replace=False):
        t = int(rng.integers(0, lv[i]))
        out.append((int(i), t))
    return A, lv, out


@pytest.mark.parametrize("seed", range(5))
def test_matches_dense_formula(seed):
    A, lv, todo = cases(seed)
    L = dense(A)
    for i, t in todo:
        row = rw.rewrite_row(A, lv, i, t)
        S = eliminated_set(A, lv, i, t)
        assert row.bcol.tolist() == S
        c = np.linalg.solve(L[np.ix_(S, S)].T, L[i, S]) if S else np.zeros(0)
        full = L[i, :i] - (c @ L[S, :i] if S else 0.0)
        X = sorted(set(np.nonzero(L[[i] + S, :i])[1].tolist()) - set(S))
        assert row.xcol.tolist() == X
        assert all(lv[k] < t for k in X)
        assert np.allclose(row.bw, c, rtol=1e-12, atol=1e-14)
        assert np.allclose(row.xval, full[X], rtol=1e-12, atol=1e-14)
        assert np.allclose(full[S], 0.0, atol=1e-12)
        assert row.diag == L[i, i]


@pytest.mark.parametrize("seed", range(3))
def test_matches_exact_rational_formula(seed):
    sympy = pytest.importorskip("sympy")
    A, lv, todo = cases(100 + seed, n=24, density=0.25, integer=True)
    L = dense(A)
    Lq = sympy.Matrix([[sympy.Rational(int(v)) for v in r] for r in L])
    for i, t in todo:
        row = rw.rewrite_row(A, lv, i, t)
        S = row.bcol.tolist()
        if not S:
            continue
        c = Lq.extract(S, S).T.LUsolve(Lq.extract([i], S).T)
        for k, w in zip(S, row.bw.tolist()):
            e = c[S.index(k)]
            assert abs(w - float(e)) <= 1e-13 * max(1.0, abs(float(e)))
        full = Lq.extract([i], list(range(i))) - c.T * Lq.extract(S, list(range(i)))
        for k, v in zip(row.xcol.tolist(), row.xval.tolist()):
            e = float(full[0, k])
            assert abs(v - e) <= 1e-13 * max(1.0, abs(e))


# --- transformed-system invariants ----------------------------------------------

@pytest.mark.parametrize("cfg,tau,d_max,rho", [
    (1, 16, 4, 0.5), (1, 10**9, 3, float("inf")), (3, 10**9, 4, 1.0),
    (2, 200, 8, 0.3)])
def test_transformed_system_invariants(cfg, tau, d_max, rho):
    A = mg.config_matrix(cfg, small=True)
    lv, nl = oracle.levels(A)
    tr = rw.transform(A, lv, nl, tau, d_max, rho, max_fill=4096)
    assert tr.nlev_new <= nl
    assert tr.added_flops <= rho * rw.total_flops(A)
    for i, row in tr.rows.items():
        assert row.diag == A.val[A.row_ptr[i + 1] - 1]
        assert all(lv[k] < row.target for k in row.xcol.tolist())
    b = mg.rhs_uniform(A.n, nrhs=2, seed=cfg)
    x = rw.solve_transformed(A, tr, b)
    assert oracle.relerr(x, oracle.forward_subst(A, b)) < 1e-12


def test_no_merge_when_nothing_is_thin():
    A = mg.config_matrix(1, small=True)
    lv, nl = oracle.levels(A)
    tr = rw.transform(A, lv, nl, tau=0, d_max=8, rho=1.0, max_fill=4096)
    assert tr.nlev_new == nl and not tr.rows


# --- selection heuristic, hand-worked -------------------------------------------

def test_selection_hand_example():
    rows = np.array([1, 1, 5, 1, 1, 1])
    cost = lambda lv, r: 10 * r
    big = 10**9
    assert rw.select_segments(rows, cost, 2, 2, 1.0, big) == [(0, 1), (2, 2), (5, 0)]
    assert rw.select_segments(rows, cost, 2, 2, 1.0, 25) == [(0, 1), (2, 1), (4, 0), (5, 0)]
    assert rw.select_segments(rows, cost, 1, 2, 1.0, big) == [(i, 0) for i in range(6)]
    capped = lambda lv, r: None if lv == 3 else 10 * r
    assert rw.select_segments(rows, capped, 2, 2, 1.0, big) == [(0, 1), (2, 0), (3, 2)]
    assert rw.select_segments(rows, cost, 2, 0, 1.0, big) == [(i, 0) for i in range(6)]


# --- the paper's worked example, as stated in the text (tests/golden) -----------

def load_fig2_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fig2_rewriting.txt")
    deps, levels, steps = {}, {}, []
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            key, rest = line.split(" ", 1)
            if key == "dependency":
                r, ds = rest.split(":")
                deps[int(r)] = [int(v) for v in ds.split()]
            elif key == "level":
                r, lv = rest.split()
                levels[int(r)] = int(lv)
            elif key == "step":
                sub, out = rest.split("->")
                x, b, lv = (part.split() for part in out.split("|"))
                steps.append(([int(v) for v in sub.split()], [int(v) for v in x],
                              [int(v) for v in b], int(lv[0])))
    return deps, levels, steps


def test_fig2_golden_structure():
    """The dependency moves the paper describes for row 3 (Sec. III): one
    substitution (row 1) leaves a dependency on row 0 and lifts row 3 one
    level; the second (row 0) leaves no dependency at all."""
    deps, levels, steps = load_fig2_golden()
    A, _ = fig2_matrix()   # rows 0, 1, 3 with exactly these dependencies (+ row 2)
    for r, ds in deps.items():
        a, e = A.row_ptr[r], A.row_ptr[r + 1] - 1
        assert A.col[a:e].tolist() == ds
    lv, _ = oracle.levels(A)
    for r, l in levels.items():
        assert lv[r] == l
    for sub, x, b, new_level in steps:
        t = new_level   # rewriting to target level t eliminates rows at levels >= t
        row = rw.rewrite_row(A, lv, 3, t)
        assert sorted(row.bcol.tolist()) == sorted(sub) == sorted(b)
        assert row.xcol.tolist() == x
        assert max([lv[j] + 1 for j in x], default=0) == new_level

"""Pins of the critical-path oracle (oracle/critpath.py): closed forms,
a hand-worked DAG, networkx's longest path, brute force over every
segmentation, and the upper-bound property of the level-set model."""
import itertools

import numpy as np
import pytest

import matgen as mg
import oracle
from oracle import critpath as cpo


def test_chain_closed_form():
    # x_i depends on x_{i-1} only, one term: f(i) = (i + 1) H + i
    for n, H in ((1, 5), (7, 3), (50, 16)):
        A = mg.chain(n, a=0.5, diag=1.0)
        cp, f = cpo.critical_path(*cpo.plain_rows(A), H)
        assert f.tolist() == [(i + 1) * H + i for i in range(n)]
        assert cp == n * H + (n - 1)


def test_hand_worked_dag():
    # 0; 1 <- 0; 2 <- 0; 3 <- {1, 2}; 4 <- 0, H = 10
    deps = [[], [0], [0], [1, 2], [0]]
    terms = [0, 1, 1, 2, 1]
    cp, f = cpo.critical_path(deps, terms, 10)
    assert f.tolist() == [10, 21, 21, 33, 21]
    assert cp == 33


def test_networkx_longest_path():
    nx = pytest.importorskip("networkx")
    for seed in range(4):
        A = mg.random_lower(70, seed=seed, density=0.1)
        H = 7 + seed
        deps, terms = cpo.plain_rows(A)
        G = nx.DiGraph()
        w = [H + t for t in terms]
        for i in range(A.n):
            G.add_edge("s", i, weight=w[i])
            for j in deps[i]:
                G.add_edge(j, i, weight=w[i])
        assert cpo.critical_path(deps, terms, H)[0] == nx.dag_longest_path_length(G)


def compositions(n, d_max):
    """Every segmentation of n levels into segments of 1..d_max+1 levels."""
    if n == 0:
        yield []
        return
    for k in range(1, min(n, d_max + 1) + 1):
        for rest in compositions(n - k, d_max):
            yield [k] + rest


def segs_of(parts):
    out, t = [], 0
    for k in parts:
        out.append((t, k - 1))
        t += k
    return out


CASES = [
    ("stencil2d_4", lambda: mg.stencil2d(4)),
    ("stencil3d_3", lambda: mg.stencil3d(3, seed=2)),
    ("chain_9", lambda: mg.chain(9, a=0.5, diag=1.0)),
    ("random_40", lambda: mg.random_lower(40, seed=5, density=0.12)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("H", [1, 6, 40])
def test_dp_equals_brute_force(name, make, H):
    A = make()
    lv, nlev = oracle.levels(A)
    assert nlev <= 12
    d_max, cap = 3, 12
    table = cpo.lift_table(A, lv, nlev, d_max, cap)
    best = None
    for parts in compositions(nlev, d_max):
        segs = segs_of(parts)
        ok = all(table.get((t + r, r)) is not None for t, d in segs for r in range(1, d + 1))
        if ok:
            v = cpo.segments_cp(segs, table, H)
            best = v if best is None else min(best, v)
    segs = cpo.select_critpath(nlev, table, H, d_max)
    assert sum(d + 1 for _, d in segs) == nlev
    assert [t for t, _ in segs] == list(itertools.accumulate([0] + [d + 1 for _, d in segs[:-1]]))
    assert cpo.segments_cp(segs, table, H) == best


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_levelset_model_bounds_the_true_critical_path(name, make):
    A = make()
    lv, nlev = oracle.levels(A)
    table = cpo.lift_table(A, lv, nlev, 3, 10**6)
    rng = np.random.default_rng(3)
    for _ in range(5):
        parts, left = [], nlev
        while left:
            k = int(rng.integers(1, min(left, 4) + 1))
            parts.append(k)
            left -= k
        segs = segs_of(parts)
        deps, terms = cpo.transformed_rows(A, lv, segs)
        cp, _ = cpo.critical_path(deps, terms, 9)
        assert cp <= cpo.segments_cp(segs, table, 9)
    # all levels kept: the level-set model of a chain is exact
    C = mg.chain(6, a=0.5, diag=1.0)
    lvc, nc = oracle.levels(C)
    tc = cpo.lift_table(C, lvc, nc, 0, 10)
    assert cpo.critical_path(*cpo.plain_rows(C), 9)[0] == \
        cpo.segments_cp([(t, 0) for t in range(nc)], tc, 9)


def test_large_hop_weight_merges_and_small_one_keeps_levels():
    """With a hop far heavier than any row the DP leaves as few new levels as
    the depth limit allows; with H = 0 merging never pays on a matrix whose
    rewritten rows grow."""
    A = mg.stencil2d(6)
    lv, nlev = oracle.levels(A)
    table = cpo.lift_table(A, lv, nlev, 2, 10**6)
    deep = cpo.select_critpath(nlev, table, 10**6, 2)
    assert len(deep) == -(-nlev // 3)
    flat = cpo.select_critpath(nlev, table, 0, 2)
    assert all(d == 0 for _, d in flat)


@pytest.mark.parametrize("seed", range(6))
def test_min_sum_segmentation_equals_brute_force(seed):
    """select_min_sum against every composition of a few levels into
    segments of 1..D levels, with random costs and random missing segments
    (a missing segment also rules out the deeper ones from its level)."""
    rng = np.random.default_rng(seed)
    nlev, D = 9, 4
    cost = rng.uniform(0.1, 3.0, (nlev, D))
    ok = rng.random((nlev, D)) > 0.2
    ok[:, 0] = True
    for t in range(nlev):           # missing at d: missing deeper too
        for d in range(1, D):
            ok[t, d] = ok[t, d] and ok[t, d - 1] and t + d < nlev
    best = None
    for parts in compositions(nlev, D - 1):
        segs = segs_of(parts)
        if all(ok[t, d] for t, d in segs):
            v = sum(cost[t, d] for t, d in segs)
            best = v if best is None else min(best, v)
    segs = cpo.select_min_sum(cost, ok)
    assert sum(d + 1 for _, d in segs) == nlev
    assert np.isclose(sum(cost[t, d] for t, d in segs), best)


def test_min_sum_ties_go_to_the_smaller_depth():
    cost = np.ones((3, 3))
    cost[0, 2] = 1.0                 # one segment of 3 levels costs 1 = one level
    ok = np.ones((3, 3), bool)
    ok[1, 2] = ok[2, 1] = ok[2, 2] = False
    assert cpo.select_min_sum(cost, ok) == [(0, 2)]
    cost[0, 2] = 3.0                 # now (0..1)(2) and (0)(1..2) tie at 2:
    assert cpo.select_min_sum(cost, ok) == [(0, 0), (1, 1)]   # level 0 keeps d = 0

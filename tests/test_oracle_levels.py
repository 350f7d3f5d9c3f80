"""Pins of the oracle's level computation (DAG_L levels, Sec. II) against
closed forms of stencil wavefronts and networkx's topological generations."""
import numpy as np
import pytest

import matgen as mg
import oracle


def wavefront_sizes(side, dims):
    """Number of grid points with coordinate sum l: convolution of indicators."""
    c = np.ones(side, dtype=np.int64)
    out = c
    for _ in range(dims - 1):
        out = np.convolve(out, c)
    return out


def test_stencil2d_levels_closed_form():
    side = 64
    A = mg.stencil2d(side)
    lv, nlev = oracle.levels(A)
    r = np.arange(A.n)
    assert nlev == 2 * side - 1 == 127
    assert np.array_equal(lv, r // side + r % side)
    ptr, perm = oracle.level_sets(lv, nlev)
    assert np.array_equal(np.diff(ptr), wavefront_sizes(side, 2))
    assert np.diff(ptr).max() == 64


def test_stencil3d_levels_closed_form():
    side = 128
    A = mg.stencil3d(side, seed=2000)
    lv, nlev = oracle.levels(A)
    r = np.arange(A.n)
    assert nlev == 3 * side - 2 == 382
    assert np.array_equal(lv, r // (side * side) + (r // side) % side + r % side)
    sizes = np.bincount(lv)
    assert np.array_equal(sizes, wavefront_sizes(side, 3))
    assert sizes.max() == 12288
    assert (sizes < 32).sum() == 14 and (sizes < 1024).sum() == 88
    assert (sizes < 4096).sum() == 180


def test_chain_has_n_levels_and_diagonal_has_one():
    assert oracle.levels(mg.chain(777))[1] == 777
    n = 50
    D = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.ones(n))
    lv, nl = oracle.levels(D)
    assert nl == 1 and not lv.any()


@pytest.mark.parametrize("seed", range(5))
def test_levels_match_networkx_generations(seed):
    nx = pytest.importorskip("networkx")
    A = mg.random_lower(120, seed=seed, density=0.04)
    G = nx.DiGraph()
    G.add_nodes_from(range(A.n))
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = int(A.col[k])
            if j != i:
                G.add_edge(j, i)
    lv, nl = oracle.levels(A)
    gens = list(nx.topological_generations(G))
    assert nl == len(gens)
    for g, nodes in enumerate(gens):
        assert all(lv[v] == g for v in nodes)


def test_explicit_zero_is_still_an_edge():
    # structural reading: a stored 0.0 off the diagonal is a dependency
    A = mg.chain(5)
    A.val[A.col != np.repeat(np.arange(5), np.diff(A.row_ptr))] = 0.0
    assert oracle.levels(A)[1] == 5


def test_thin_tail_small_structure():
    A = mg.thin_tail(20_000, seed=3000)
    lv, nl = oracle.levels(A)
    n_chain = 1000
    # the chain rows are serial: each one level below the previous one
    tail = lv[-n_chain:]
    assert np.all(np.diff(tail) == 1)
    assert nl == tail[-1] + 1

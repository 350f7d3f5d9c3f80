"""Pins of the per-level feature oracle (oracle/features.py): a 3x3 grid
worked by hand, the log2 bins, stencil closed forms, the fill cap, and the
lift columns against the added FLOPs of the oracle's own transformation."""
import numpy as np

import matgen as mg
import oracle
from oracle import features as fo
from oracle import rewrite as rw


def test_hand_worked_3x3_grid():
    # levels i + j of the 5-point lower triangle on a 3x3 grid; see the
    # module docstring for the columns (bins 3..7 are empty here)
    A = mg.stencil2d(3)
    lv, nlev = oracle.levels(A)
    f = fo.level_features(A, lv, nlev, lifts=2, cap=10**6)
    expect = [
        # rows nnz b0 b1 b2 span lift1 lift2
        [1, 0, 1, 0, 0, 0, 0, 0],
        [2, 2, 0, 2, 0, 1, 0, 0],
        [3, 4, 0, 2, 1, 1, 6, 6],
        [2, 4, 0, 0, 2, 1, 8, 12],
        [1, 2, 0, 0, 1, 1, 6, 10],
    ]
    got = np.concatenate([f[:, :5], f[:, 10:13]], axis=1)
    assert got.tolist() == expect
    assert not f[:, 5:10].any()


def test_log2_bins():
    cases = {0: 0, 1: 1, 2: 2, 3: 2, 4: 3, 7: 3, 8: 4, 31: 5, 32: 6, 63: 6, 64: 7, 5000: 7}
    for c, b in cases.items():
        assert fo.length_bin(c) == b


def test_stencil3d_closed_forms():
    s = 6
    A = mg.stencil3d(s, seed=1)
    lv, nlev = oracle.levels(A)
    f = fo.level_features(A, lv, nlev, lifts=0, cap=10**6)
    # rows per level: number of (i, j, k) in [0, s)^3 with i + j + k = l
    rows = np.convolve(np.convolve(np.ones(s), np.ones(s)), np.ones(s))
    assert f[:, 0].tolist() == rows.tolist()
    # every stored off-diagonal entry is counted once, in its row's level
    assert f[:, 1].sum() == A.nnz - A.n
    assert (f[:, 2:10].sum(axis=1) == f[:, 0]).all()
    # a 7-point row has at most 3 dependencies: bins 0..2 only, span 1
    assert not f[:, 5:10].any()
    assert f[1:, 10].tolist() == [1.0] * (nlev - 1) and f[0, 10] == 0


def test_fill_cap_marks_the_lift():
    A = mg.stencil2d(5)
    lv, nlev = oracle.levels(A)
    f = fo.level_features(A, lv, nlev, lifts=2, cap=3)
    assert (f[:, 11:] == -1).any()
    assert ((f[:, 11:] >= -1)).all()


def test_lifts_sum_to_the_transform_added_flops():
    A = mg.random_lower(120, seed=4, density=0.06)
    lv, nlev = oracle.levels(A)
    d = 2
    f = fo.level_features(A, lv, nlev, lifts=d, cap=10**6)
    tr = rw.transform(A, lv, nlev, tau=10**9, d_max=d, rho=float("inf"), max_fill=10**6)
    tot = 0
    for t, dd in tr.segments:
        for r in range(1, dd + 1):
            tot += f[t + r, 10 + r]
    assert tot == tr.added_flops

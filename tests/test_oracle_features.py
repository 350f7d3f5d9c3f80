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


def test_segment_features_hand_worked_3x3_grid():
    """Segments of the 3x3 grid worked by hand (nnz = 21 with the diagonal).
    (0, 1): rows 3, terms 0 + 2 (level 1's entries; lifting it onto level
    0 trades each x00 term for a b00 term: +0), the longest row 1 term.
    (0, 2): rows 6; level 2 lifted by 2 adds 6 FLOPs = 3 terms, so terms
    0 + 2 + 4 + 3 = 9; its longest row is (1,1) with b01, b10, b00."""
    A = mg.stencil2d(3)
    lv, nlev = oracle.levels(A)
    f, ok = fo.segment_features(A, lv, nlev, d_max=2, cap=10**6)
    ln, ld = np.log2(9), np.log2(21 / 9)
    np.testing.assert_allclose(f[0, 0], [1, 0, 0, 0, 0, 0, ln, ld])
    np.testing.assert_allclose(f[0, 1], [2, np.log2(3), 1, 2 / 3, 1, 2 / 3, ln, ld])
    np.testing.assert_allclose(f[0, 2], [np.log2(7), np.log2(10), 2, 1.5, 2, 5 / 6, ln, ld])
    assert ok[:3].all() and ok[3].tolist() == [True, True, False]
    assert ok[4].tolist() == [True, False, False]
    # a cap of 2 terms rules out lifting level 2 by 2 ((1,1) needs 3)
    _, ok2 = fo.segment_features(A, lv, nlev, d_max=2, cap=2)
    assert ok2[0].tolist() == [True, True, False]


def test_segment_features_invariants():
    A = mg.random_lower(60, seed=3, density=0.08)
    lv, nlev = oracle.levels(A)
    f, ok = fo.segment_features(A, lv, nlev, d_max=3, cap=10**6)
    base = fo.level_features(A, lv, nlev, 3, 10**6)
    rows = np.exp2(f[..., 0]) - 1
    terms = np.exp2(f[..., 1]) - 1
    # d = 0: the level itself
    np.testing.assert_allclose(rows[:, 0], base[:, 0])
    np.testing.assert_allclose(terms[:, 0], base[:, 1])
    assert (f[:, :, 4][ok] == np.broadcast_to(np.arange(4), ok.shape)[ok]).all()
    # merging never loses a row or a term, and rewrites at least the lifted rows
    for t in range(nlev):
        for d in range(1, 4):
            if ok[t, d]:
                assert np.isclose(rows[t, d], rows[t, d - 1] + base[t + d, 0])
                assert terms[t, d] >= terms[t, d - 1] + base[t + d, 1] - 1e-9
                assert f[t, d, 5] > 0
    # a segmentation into feasible segments covers every row once
    t, total = 0, 0.0
    while t < nlev:
        d = max(k for k in range(4) if ok[t, k])
        total += rows[t, d]
        t += d + 1
    assert np.isclose(total, A.n)

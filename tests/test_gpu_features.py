"""GPU parity of the per-level features (sptrsv_level_features) against the
oracle (oracle/features.py): every column equal on small matrices of each
family, and at the full 128^3 size the closed forms of the stencil."""
import numpy as np
import pytest

import matgen as mg
import oracle
from gpu_util import plan_for
from oracle import features as fo

pytestmark = pytest.mark.gpu

MATS = [
    ("stencil2d_3", lambda: mg.stencil2d(3)),
    ("stencil2d_20", lambda: mg.stencil2d(20)),
    ("stencil3d_8", lambda: mg.stencil3d(8, seed=2)),
    ("random_400", lambda: mg.random_lower(400, seed=7, density=0.04)),
    ("thin_tail_3000", lambda: mg.thin_tail(3000, seed=5)),
]


@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
@pytest.mark.parametrize("lifts,cap", [(0, 1024), (2, 1024), (3, 40)])
def test_level_features_match_oracle(name, make, lifts, cap):
    from paper_2103_11445_gb300 import binding as B
    A = make()
    lv, nlev = oracle.levels(A)
    P = plan_for(A, select_mode=0, solve_mode=2, max_row_fill=cap)
    got = B.sptrsv_level_features(P.handle, nlev, lifts)
    ref = fo.level_features(A, lv, nlev, lifts, cap)
    assert np.array_equal(got.astype(np.float64), ref)
    P.close()


def test_long_rows_fill_the_last_bin():
    """Rows of 70 dependencies land in bin 7 (>= 64); no lift columns (the
    oracle's Python rewriting of such rows would take minutes)."""
    from paper_2103_11445_gb300 import binding as B
    A = mg.banded(3000, seed=8, band=2000, per_row=70)
    lv, nlev = oracle.levels(A)
    P = plan_for(A, select_mode=0, solve_mode=2)
    got = B.sptrsv_level_features(P.handle, nlev, 0)
    ref = fo.level_features(A, lv, nlev, 0, 1024)
    assert np.array_equal(got.astype(np.float64), ref)
    assert ref[:, 9].sum() > 0
    P.close()


def test_full_stencil3d_closed_forms():
    from paper_2103_11445_gb300 import binding as B
    s = 128
    A = mg.stencil3d(s, seed=2000)
    P = plan_for(A, select_mode=0, solve_mode=2)
    f = B.sptrsv_level_features(P.handle, 382, 1).astype(np.float64)
    rows = np.convolve(np.convolve(np.ones(s), np.ones(s)), np.ones(s))
    assert np.array_equal(f[:, 0], rows)
    assert f[:, 1].sum() == A.nnz - A.n
    assert np.array_equal(f[:, 2:10].sum(axis=1), rows)
    assert f[0, 10] == 0 and (f[1:, 10] == 1).all()
    # lifting level 1 (rows on the source row only) adds no term; every
    # later level gains some
    assert (f[2:, 11] > 0).all() and f[0, 11] == 0 and f[1, 11] == 0
    P.close()

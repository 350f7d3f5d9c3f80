"""GPU parity of the level analysis (validation, levels, level-ordered
permutation) against the oracle: integer outputs must match bit for bit."""
import numpy as np
import pytest

import matgen as mg
import oracle
from gpu_util import plan_for

pytestmark = pytest.mark.gpu


def check_levels(A):
    P = plan_for(A)
    lv, lp, pm = (t.cpu().numpy() for t in P.levels())
    ref_lv, ref_n = oracle.levels(A)
    ref_lp, ref_pm = oracle.level_sets(ref_lv, ref_n)
    info = P.info()
    assert info["nlev"] == ref_n
    assert np.array_equal(lv, ref_lv)
    assert np.array_equal(lp, ref_lp)
    assert np.array_equal(pm, ref_pm)
    P.close()
    return ref_n


@pytest.mark.parametrize("name,make", [
    ("stencil2d_64", lambda: mg.stencil2d(64)),
    ("stencil3d_16", lambda: mg.stencil3d(16, seed=1)),
    ("thin_tail_20k", lambda: mg.thin_tail(20_000, seed=3)),
    ("random_300", lambda: mg.random_lower(300, seed=5, density=0.05)),
    ("chain_5000", lambda: mg.chain(5000)),
    ("banded_70k", lambda: mg.banded(70_000, seed=11)),
])
def test_levels_match_oracle(name, make):
    check_levels(make())


def test_levels_full_stencil3d_128():
    assert check_levels(mg.stencil3d(128, seed=2000)) == 382


def test_levels_full_thin_tail():
    check_levels(mg.thin_tail(1_000_000, seed=3000))


def test_diagonal_and_single_row():
    n = 1000
    D = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.full(n, 2.0))
    assert check_levels(D) == 1
    one = mg.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    assert check_levels(one) == 1


def test_empty_matrix():
    from paper_2103_11445_gb300 import binding as B
    import torch
    h = B.sptrsv_analyze(0, 0, 0, 0, 0, 0)
    info = B.sptrsv_get_info(h)
    assert info.n == 0 and info.nlev == 0
    b = torch.zeros(0, dtype=torch.float64, device="cuda")
    B.sptrsv_solve(h, 0, 0, 1, 0)
    B.sptrsv_plan_destroy(h)


@pytest.mark.parametrize("mutate,code", [
    ("unsorted", 3), ("upper", 2), ("missing_diag", 5), ("zero_diag", 4), ("bad_ptr", 3),
])
def test_invalid_csr_rejected(mutate, code):
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(8)
    rp, col, val = A.row_ptr.copy(), A.col.copy(), A.val.copy()
    i = 20
    a, e = rp[i], rp[i + 1]
    if mutate == "unsorted":
        col[a], col[a + 1] = col[a + 1], col[a]
    elif mutate == "upper":
        col[e - 1] = i + 1
    elif mutate == "zero_diag":
        val[e - 1] = 0.0
    elif mutate == "bad_ptr":
        rp[i + 1] = rp[i] - 1
    if mutate == "missing_diag":
        # drop the diagonal of row i entirely
        keep = np.ones(col.size, bool)
        keep[e - 1] = False
        col, val = col[keep], val[keep]
        rp = rp.copy()
        rp[i + 1:] -= 1
    with pytest.raises(B.SptrsvError) as ei:
        B.Plan(A.n, rp, col, val)
    assert ei.value.code == code

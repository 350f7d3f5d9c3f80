"""GPU parity of the critical-path-driven selection (SELECT_CRITPATH) and of
the device's weighted critical path (sptrsv_critical_path) against the
oracle (oracle/critpath.py): critical paths of plain and rewritten
structures equal the oracle's exactly, the selected segments equal the
oracle's dynamic programme exactly, and at the full 128^3 size the selection
is optimal among the fixed depths it could have taken."""
import numpy as np
import pytest

import matgen as mg
import oracle
from gpu_util import assert_close_to_oracle, gpu_solve, plan_for
from oracle import critpath as cpo

pytestmark = pytest.mark.gpu

MATS = [
    ("stencil2d_16", lambda: mg.stencil2d(16)),
    ("stencil3d_9", lambda: mg.stencil3d(9, seed=4)),
    ("random_300", lambda: mg.random_lower(300, seed=6, density=0.03)),
    ("thin_tail_4000", lambda: mg.thin_tail(4000, seed=12)),
    ("chain_400", lambda: mg.chain(400, a=0.5, diag=1.0)),
]
SELECTIONS = [
    ("plain", dict(select_mode=0)),
    ("fixed_d2", dict(select_mode=3, depth=2)),
    ("heuristic", dict(select_mode=1)),
    ("critpath", dict(select_mode=5, max_depth=3, hop_weight=12)),
]


@pytest.mark.parametrize("sname,kw", SELECTIONS, ids=[s[0] for s in SELECTIONS])
@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
@pytest.mark.parametrize("H", [1, 16])
def test_device_critical_path_matches_oracle(name, make, sname, kw, H):
    from paper_2103_11445_gb300 import binding as B
    A = make()
    P = plan_for(A, solve_mode=2, **kw)
    lv, _ = oracle.levels(A)
    first, depth = P.segments()
    segs = list(zip(first, depth))
    deps, terms = cpo.transformed_rows(A, lv, segs)
    assert B.sptrsv_critical_path(P.handle, H) == cpo.critical_path(deps, terms, H)[0]
    P.close()


SEL_MATS = [
    ("stencil2d_12", lambda: mg.stencil2d(12)),
    ("stencil3d_6", lambda: mg.stencil3d(6, seed=3)),
    ("random_200", lambda: mg.random_lower(200, seed=9, density=0.05)),
    ("thin_tail_3000", lambda: mg.thin_tail(3000, seed=21)),
]


@pytest.mark.parametrize("name,make", SEL_MATS, ids=[m[0] for m in SEL_MATS])
@pytest.mark.parametrize("H,d_max,cap", [(4, 3, 1024), (16, 3, 1024), (64, 4, 24)])
def test_selection_matches_oracle(name, make, H, d_max, cap):
    A = make()
    lv, nlev = oracle.levels(A)
    table = cpo.lift_table(A, lv, nlev, d_max, cap)
    ref = cpo.select_critpath(nlev, table, H, d_max)
    P = plan_for(A, select_mode=5, hop_weight=H, max_depth=d_max, max_row_fill=cap,
                 solve_mode=2)
    first, depth = P.segments()
    assert list(zip(first, depth)) == ref
    b = mg.rhs_uniform(A.n, seed=2)
    assert_close_to_oracle(A, gpu_solve(P, b), b, 1e-10)
    P.close()


def levelset_cp(P, H):
    """sum over new levels of H + most terms of a row in it, from the
    exported transformed rows"""
    t = P.transformed()
    nl = t["new_level"].cpu().numpy()
    terms = (np.diff(t["xptr"].cpu().numpy()) + np.diff(t["bptr"].cpu().numpy()))
    m = np.zeros(nl.max() + 1, np.int64)
    np.maximum.at(m, nl, terms)
    return int((H + m).sum())


def test_full_stencil3d_selection_is_optimal_among_fixed_depths():
    A = mg.stencil3d(128, seed=2000)
    H = 16
    P = plan_for(A, select_mode=5, hop_weight=H, max_depth=4, solve_mode=2)
    best = levelset_cp(P, H)
    for d in range(0, 5):
        Q = plan_for(A, select_mode=3, depth=d, solve_mode=2)
        assert best <= levelset_cp(Q, H), d
        Q.close()
    b = mg.rhs_uniform(A.n, seed=2001)
    assert_close_to_oracle(A, gpu_solve(P, b), b, 1e-10)
    P.close()

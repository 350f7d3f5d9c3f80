"""GPU parity of the equation-rewriting transform (Sec. III) against the
oracle: the chosen new levels (integers, exact), every rewritten row's
pattern (exact) and coefficients (FP64, relative 1e-12), and the solution of
the transformed system (relerr <= 1e-10)."""
import numpy as np
import pytest

import matgen as mg
import oracle
from oracle import rewrite as rw
from gpu_util import assert_close_to_oracle, gpu_solve, plan_for

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
COEF_RTOL = 1e-12


def oracle_transform(A, tau, d_max, rho, cap=1024):
    lv, nl = oracle.levels(A)
    return rw.transform(A, lv, nl, tau, d_max, rho, cap)


def exported(P, A):
    t = {k: v.cpu().numpy() for k, v in P.transformed().items()}
    return t


def compare_rows(A, tr, t, rows):
    for i in rows:
        x0, x1 = t["xptr"][i], t["xptr"][i + 1]
        b0, b1 = t["bptr"][i], t["bptr"][i + 1]
        if i in tr.rows:
            ref = tr.rows[i]
            xc, xv, bc, bw = ref.xcol, ref.xval, ref.bcol, ref.bw
        else:
            a, e = A.row_ptr[i], A.row_ptr[i + 1] - 1
            xc, xv = A.col[a:e], A.val[a:e]
            bc, bw = np.zeros(0, np.int32), np.zeros(0)
        assert np.array_equal(t["xcol"][x0:x1], xc), i
        assert np.array_equal(t["bcol"][b0:b1], bc), i
        scale = max(1.0, np.abs(np.concatenate([xv, bw])).max(initial=0.0))
        assert np.allclose(t["xval"][x0:x1], xv, rtol=COEF_RTOL, atol=COEF_RTOL * scale), i
        assert np.allclose(t["bw"][b0:b1], bw, rtol=COEF_RTOL, atol=COEF_RTOL * scale), i


CASES = [
    ("stencil2d_64", lambda: mg.stencil2d(64), 16, 4, 0.5),
    ("stencil2d_64_all", lambda: mg.stencil2d(64), 10**9, 3, float("inf")),
    ("stencil3d_16", lambda: mg.stencil3d(16, seed=1), 200, 8, 0.3),
    ("thin_tail_20k", lambda: mg.thin_tail(20_000, seed=3000), 10**9, 4, 1.0),
    ("thin_tail_20k_h", lambda: mg.thin_tail(20_000, seed=3000), 40, 8, 0.1),
    ("random_400", lambda: mg.random_lower(400, seed=9, density=0.02), 10**9, 3, 2.0),
]


@pytest.mark.parametrize("name,make,tau,d_max,rho", CASES, ids=[c[0] for c in CASES])
def test_heuristic_matches_oracle(name, make, tau, d_max, rho):
    A = make()
    tr = oracle_transform(A, tau, d_max, rho)
    budget = rho if np.isfinite(rho) else 1e300
    P = plan_for(A, select_mode=1, thin_rows=min(tau, 2**31 - 1), max_depth=d_max,
                 flop_budget=budget, max_row_fill=1024, solve_mode=1)
    info = P.info()
    first, depth = P.segments()
    assert list(zip(first, depth)) == tr.segments
    assert info["nlev_new"] == tr.nlev_new <= info["nlev"]
    assert info["rows_rewritten"] == len(tr.rows)
    t = exported(P, A)
    assert np.array_equal(t["new_level"], tr.new_level)
    compare_rows(A, tr, t, range(A.n))
    assert info["flops_new"] - info["flops_plain"] == tr.added_flops
    b = mg.rhs_uniform(A.n, nrhs=2, seed=5)
    for mode in (dict(solve_mode=1), dict(solve_mode=2)):
        P.transform(select_mode=1, thin_rows=min(tau, 2**31 - 1), max_depth=d_max,
                    flop_budget=budget, max_row_fill=1024, **mode)
        assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)


@pytest.mark.parametrize("d", [1, 2, 3, 7])
def test_fixed_depth_chain_closed_form(d):
    m, a = 200, 0.5
    A = mg.chain(m, a=a, diag=1.0)
    P = plan_for(A, select_mode=3, depth=d, solve_mode=1)
    assert P.info()["nlev_new"] == -(-m // (d + 1))
    t = exported(P, A)
    for i in range(m):
        tgt = (i // (d + 1)) * (d + 1)
        r = i - tgt
        x0, x1 = t["xptr"][i], t["xptr"][i + 1]
        b0, b1 = t["bptr"][i], t["bptr"][i + 1]
        if r == 0:
            assert list(t["xcol"][x0:x1]) == ([i - 1] if i else [])
            assert b1 == b0
            continue
        if tgt == 0:
            assert x1 == x0
        else:
            assert list(t["xcol"][x0:x1]) == [tgt - 1]
            assert t["xval"][x0] == -(a ** (r + 1))
        assert list(t["bcol"][b0:b1]) == list(range(tgt, i))
        assert list(t["bw"][b0:b1]) == [-(a ** (i - j)) for j in range(tgt, i)]
    b = mg.rhs_uniform(m, seed=1)
    assert_close_to_oracle(A, gpu_solve(P, b), b, 1e-15)


def test_fig2_example_on_device():
    l00, l10, l11, l20, l22, l31, l33 = 2.0, 0.5, 4.0, -1.0, 8.0, 3.0, 0.25
    A = mg.CSR(4, np.array([0, 1, 3, 5, 7], np.int32), np.array([0, 0, 1, 0, 2, 1, 3], np.int32),
               np.array([l00, l10, l11, l20, l22, l31, l33]))
    P = plan_for(A, select_mode=3, depth=2, solve_mode=1)
    t = exported(P, A)
    b0, b1 = t["bptr"][3], t["bptr"][4]
    assert t["xptr"][4] == t["xptr"][3]
    assert list(t["bcol"][b0:b1]) == [0, 1]
    assert t["bw"][b0 + 1] == l31 / l11
    assert t["bw"][b0] == -(l31 * l10) / (l11 * l00)


@pytest.mark.parametrize("mode", [1, 2], ids=["barrier", "syncfree"])
@pytest.mark.parametrize("d", [1, 3])
def test_full_stencil3d_fixed_depth(mode, d):
    A = mg.stencil3d(128, seed=2000)
    P = plan_for(A, select_mode=3, depth=d, solve_mode=mode)
    info = P.info()
    assert info["nlev_new"] == -(-382 // (d + 1))
    b = mg.rhs_uniform(A.n, seed=2001)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)
    # sampled rewritten rows against the oracle, one by one
    lv, _ = oracle.levels(A)
    t = exported(P, A)
    rng = np.random.default_rng(d)
    for i in rng.choice(A.n, 300, replace=False).tolist():
        tgt = (int(lv[i]) // (d + 1)) * (d + 1)
        x0, x1 = t["xptr"][i], t["xptr"][i + 1]
        b0, b1 = t["bptr"][i], t["bptr"][i + 1]
        if tgt == lv[i]:
            assert b1 == b0
            continue
        ref = rw.rewrite_row(A, lv, i, tgt)
        assert np.array_equal(t["xcol"][x0:x1], ref.xcol)
        assert np.array_equal(t["bcol"][b0:b1], ref.bcol)
        assert np.allclose(t["xval"][x0:x1], ref.xval, rtol=COEF_RTOL, atol=1e-15)
        assert np.allclose(t["bw"][b0:b1], ref.bw, rtol=COEF_RTOL, atol=1e-15)


@pytest.mark.parametrize("mode", [1, 2], ids=["barrier", "syncfree"])
def test_full_thin_tail_depth_sweep(mode):
    A = mg.thin_tail(1_000_000, seed=3000)
    b = mg.rhs_uniform(A.n, seed=3001)
    ref = oracle.forward_subst(A, b)
    prev = None
    for d in (1, 4, 8):
        P = plan_for(A, select_mode=3, depth=d, solve_mode=mode)
        nl = P.info()["nlev_new"]
        assert prev is None or nl < prev
        prev = nl
        assert oracle.relerr(gpu_solve(P, b), ref) <= TOL64
        P.close()


def test_autotuned_transform_solves():
    A = mg.stencil3d(40, seed=2)
    P = plan_for(A, select_mode=3, depth=2, solve_mode=0)
    b = mg.rhs_uniform(A.n, nrhs=3, seed=2)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)
    P.transform(select_mode=3, depth=2, solve_mode=0, precision=1)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)


def test_fill_cap_stops_merging():
    A = mg.stencil3d(16, seed=1)
    tr = oracle_transform(A, 10**9, 8, float("inf"), cap=12)
    P = plan_for(A, select_mode=1, thin_rows=2**31 - 1, max_depth=8, flop_budget=1e300,
                 max_row_fill=12, solve_mode=1)
    first, depth = P.segments()
    assert list(zip(first, depth)) == tr.segments
    assert max(r.fill for r in tr.rows.values()) <= 12


def test_autotune_cache_reuses_the_launch_for_the_same_shape():
    from paper_2103_11445_gb300 import binding as B
    B.sptrsv_autotune_cache_clear()
    A = mg.stencil3d(24, seed=8)
    P = plan_for(A, select_mode=3, depth=2)          # SOLVE_AUTO: timed
    i1 = P.info()
    assert i1["tuned_from_cache"] == 0
    Q = plan_for(A, select_mode=3, depth=2)          # same shape: cached
    i2 = Q.info()
    assert i2["tuned_from_cache"] == 1
    for k in ("solve_mode", "lanes_per_row", "block_threads", "grid_blocks", "cta_run_rows",
              "poll_backoff_ns"):
        assert i1[k] == i2[k], k
    assert i2["transform_ms"] < i1["transform_ms"]
    b = mg.rhs_uniform(A.n, seed=3)
    assert_close_to_oracle(A, gpu_solve(Q, b), b, TOL64)
    P.transform(select_mode=3, depth=3)              # another shape: timed again
    assert P.info()["tuned_from_cache"] == 0
    B.sptrsv_autotune_cache_clear()
    P.transform(select_mode=3, depth=2)
    assert P.info()["tuned_from_cache"] == 0


def test_select_auto_keeps_a_timed_candidate():
    """SELECT_AUTO times its candidates inside sptrsv_transform and keeps one
    of them: the plan's segments are those of the candidate it names, and
    the solve matches the oracle."""
    A = mg.stencil3d(24, seed=8)
    P = plan_for(A, select_mode=4, solve_mode=2)
    info = P.info()
    assert info["select_mode"] == 4
    code = info["chosen_depth"]
    assert code in (0, 1, 2, 3, 200, 108, 116, 300)
    if code == 0:
        kw = dict(select_mode=0)
    elif code == 300:
        kw = dict(select_mode=5, max_depth=4)
    elif code == 200:
        kw = dict(select_mode=1)
    elif code >= 100:
        kw = dict(select_mode=1, thin_rows=32, max_depth=code - 100, flop_budget=4.0)
    else:
        kw = dict(select_mode=3, depth=code)
    Q = plan_for(A, solve_mode=2, **kw)
    assert P.segments() == Q.segments()
    b = mg.rhs_uniform(A.n, seed=9)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)

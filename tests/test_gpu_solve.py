"""GPU parity of the plain level-set solves (barrier and synchronisation-free,
every lane layout, one and several right-hand sides, FP64 and FP32 with FP64
refinement) against the oracle, plus closed forms, edge cases and the
bounded-wait failure path."""
import numpy as np
import pytest

import matgen as mg
import oracle
from gpu_util import assert_close_to_oracle, gpu_solve, plan_for

pytestmark = pytest.mark.gpu

TOL64 = 1e-10   # relerr bound for FP64 results
TOL32 = 1e-5    # relerr bound for unrefined FP32 results

B_MODES = [dict(solve_mode=1, cta_run_rows=-1), dict(solve_mode=1, cta_run_rows=0),
           dict(solve_mode=2), dict(solve_mode=2, stage_z=-1)]
B_IDS = ["barrier", "barrier_runs", "syncfree", "syncfree_unstaged"]


def plain(**kw):
    d = dict(select_mode=0)
    d.update(kw)
    return d


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
@pytest.mark.parametrize("L", [1, 2, 4, 8, 32])
def test_modes_and_layouts(mode, L):
    A = mg.thin_tail(20_000, seed=3)
    P = plan_for(A, **plain(lanes_per_row=L, **mode))
    b = mg.rhs_uniform(A.n, seed=1)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
@pytest.mark.parametrize("nrhs", [2, 3, 8, 32, 33, 40])
def test_multi_rhs(mode, nrhs):
    A = mg.stencil3d(12, seed=4)
    P = plan_for(A, **plain(**mode))
    b = mg.rhs_uniform(A.n, nrhs=nrhs, seed=nrhs)
    x = gpu_solve(P, b)
    assert x.shape == b.shape
    assert_close_to_oracle(A, x, b, TOL64)


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
@pytest.mark.parametrize("hint,nrhs", [(4, 3), (8, 8), (32, 32), (32, 5), (2, 40)])
def test_multi_rhs_layout_hint(mode, hint, nrhs):
    """A structure laid out for `hint` columns (nrhs_hint), rewritten, solved
    with nrhs columns (the hint is only a layout choice)."""
    A = mg.thin_tail(6000, seed=77)
    P = plan_for(A, select_mode=3, depth=2, nrhs_hint=hint, **mode)
    L = 1
    while L < hint:
        L *= 2
    assert P.info()["lanes_per_row"] == L
    b = mg.rhs_uniform(A.n, nrhs=nrhs, seed=hint)
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
def test_closed_forms(mode):
    n = 3000
    ident = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    b = mg.rhs_uniform(n, seed=2)
    assert np.array_equal(gpu_solve(plan_for(ident, **plain(**mode)), b), b)
    d = np.random.default_rng(1).uniform(0.5, 4.0, n)
    diag = mg.CSR(n, ident.row_ptr, ident.col, d)
    assert np.array_equal(gpu_solve(plan_for(diag, **plain(**mode)), b), b / d)
    chain = mg.chain(n, a=1.0, diag=1.0)
    x = gpu_solve(plan_for(chain, **plain(**mode)), np.ones(n))
    assert np.array_equal(x, np.arange(1, n + 1, dtype=np.float64))


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
def test_diagonal_division_is_correctly_rounded(mode):
    """x_i = b_i / d_i must be the IEEE quotient bit for bit over the whole
    exponent range, zeros, subnormals, infinities and NaN included."""
    rng = np.random.default_rng(11)
    n = 200_000
    d = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-1060, 1060, n))
    b = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-1074, 1023, n))
    d[:8] = [1.0, -3.0, 5e-324, 2.0 ** -1000, 2.0 ** 1000, 1.7e308, -4.9e-324, 0.1]
    b[:8] = [0.0, -0.0, 1.0, np.inf, -np.inf, np.nan, 3.0, 5e-324]
    d = np.where(d == 0.0, 1.0, d)
    A = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    with np.errstate(all="ignore"):
        ref = b / d
    x = gpu_solve(plan_for(A, **plain(**mode)), b)
    same = (x.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(x) & np.isnan(ref))
    assert same.all(), np.nonzero(~same)[0][:10]


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
def test_random_small_matrices(mode):
    for seed in range(4):
        A = mg.random_lower(257, seed=seed, density=0.08)
        b = mg.rhs_uniform(A.n, nrhs=2, seed=seed)
        assert_close_to_oracle(A, gpu_solve(plan_for(A, **plain(**mode)), b), b, TOL64)


def test_single_row_and_long_rows():
    one = mg.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    assert gpu_solve(plan_for(one, **plain(solve_mode=2)), np.array([2.0]))[0] == 0.5
    # a row with 5000 dependencies exercises wide chunks and 32-lane rows
    n = 6000
    cols = [np.zeros(0, np.int64)] * (n - 1) + [np.arange(n - 1 - 5000, n - 1)]
    vals = [np.zeros(0)] * (n - 1) + [np.full(5000, 1e-4)]
    A = mg._from_row_lists(n, cols, vals, np.full(n, 2.0))
    b = mg.rhs_uniform(n, seed=3)
    for L in (1, 32):
        for mode in B_MODES:
            x = gpu_solve(plan_for(A, **plain(lanes_per_row=L, **mode)), b)
            assert_close_to_oracle(A, x, b, TOL64)


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16])
def test_staged_slots_of_few_long_rows(L):
    """Three levels of one long row each (70, 40 and 20 dependencies, nearly
    all on a 4096-row level just before): each forms a one-row chunk that fits
    a staging slot however wide it is, so its late terms go every way the
    staged kernel has -- deferred to the row's first lane (up to 64
    lane-steps), to every lane (more), or waited for on the spot (a chunk
    wider than 32 steps)."""
    rng = np.random.default_rng(40 + L)
    w = 4096
    n = 2 * w + 3 + 200
    cols, vals = [], []
    for i in range(n):
        if i < w:
            c = np.zeros(0, np.int64)
        elif i < 2 * w:
            c = np.array([i - w], np.int64)
        elif i < 2 * w + 3:
            k = i - 2 * w
            c = rng.choice(np.arange(w, 2 * w), (70, 39, 19)[k], replace=False)
            c = np.sort(np.concatenate([c, np.arange(2 * w, i)]))
        else:
            c = np.array([i - 3, i - 1], np.int64)
        cols.append(c.astype(np.int64))
        vals.append(rng.uniform(-1, 1, c.size) / max(1, c.size))
    A = mg._from_row_lists(n, cols, vals, 1.5 + rng.uniform(0, 1, n))
    lv, _ = oracle.levels(A)
    assert [int(lv[2 * w + k]) for k in range(3)] == [2, 3, 4]
    P = plan_for(A, **plain(solve_mode=2, lanes_per_row=L))
    assert P.info()["stage_z"] > 0
    for seed in range(3):
        b = mg.rhs_uniform(n, seed=seed)
        assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
def test_full_stencil3d_128(mode):
    A = mg.stencil3d(128, seed=2000)
    b = mg.rhs_uniform(A.n, seed=2001)
    assert_close_to_oracle(A, gpu_solve(plan_for(A, **plain(**mode)), b), b, TOL64)


@pytest.mark.parametrize("mode", B_MODES, ids=B_IDS)
def test_full_thin_tail(mode):
    A = mg.thin_tail(1_000_000, seed=3000)
    b = mg.rhs_uniform(A.n, seed=3001)
    assert_close_to_oracle(A, gpu_solve(plan_for(A, **plain(**mode)), b), b, TOL64)


def test_manufactured_stencil2d():
    A = mg.stencil2d(64)
    x_true = np.random.default_rng(1000).uniform(-1, 1, A.n)
    b = mg.manufactured_rhs(A, x_true)
    x = gpu_solve(plan_for(A), b)
    assert oracle.relerr(x, x_true) < 1e-12
    assert_close_to_oracle(A, x, b, TOL64)


@pytest.mark.parametrize("mode", [1, 2], ids=["barrier", "syncfree"])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_fp32_with_refinement(mode, nrhs):
    A = mg.thin_tail(20_000, seed=7)
    b = mg.rhs_uniform(A.n, nrhs=nrhs, seed=8)
    P = plan_for(A, **plain(solve_mode=mode, precision=1))
    assert_close_to_oracle(A, gpu_solve(P, b), b, TOL64)
    assert P.info()["ir_iters_last"] >= 1
    P0 = plan_for(A, **plain(solve_mode=mode, precision=1, ir_max_iter=0))
    err = assert_close_to_oracle(A, gpu_solve(P0, b), b, TOL32)
    assert err > 1e-12  # really computed in FP32


def test_aliasing_rejected():
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(8)
    P = plan_for(A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SptrsvError) as ei:
        P.solve(b, b)
    assert ei.value.code == 1


def test_syncfree_wait_times_out_and_latches():
    """A row made to wait on its own unknown can never be satisfied: the
    bounded spin must give up, report TIMEOUT and leave the device usable."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(32)
    P = plan_for(A, **plain(solve_mode=2, wait_timeout_ms=200))
    B.sptrsv_debug_inject_wait(P.handle, A.n - 1)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    P.solve(b)
    code = B.sptrsv_check(P.handle, 0)
    assert code == 8  # SPTRSV_ERR_TIMEOUT
    with pytest.raises(B.SptrsvError) as ei:
        P.solve(b)
    assert ei.value.code == 9  # BAD_STATE
    P.close()
    # the context is still healthy: a fresh plan solves correctly
    bb = mg.rhs_uniform(A.n, seed=1)
    assert_close_to_oracle(A, gpu_solve(plan_for(A, **plain(solve_mode=2)), bb), bb, TOL64)

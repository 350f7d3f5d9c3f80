"""GPU parity of the single-CTA tail (transform parameter tail_rows): the
trailing levels of at most tail_rows rows are solved by one CTA after the
main kernel, with the terms from before them folded into one constant per
row by a grid-wide pre-pass.  Every case is compared with the oracle's
substitution for its operator; the cases span a tail that is the whole
matrix (a chain), tails after a grid-wide part (stencils, the thin-tail
matrix), in-tail terms read from the shared-memory window and from x (the
full 1M-row matrix, whose tail reaches back further than the window), rows
with up to 16 in-tail terms, both main kernels, and the operators solved
through a mirrored structure."""
import numpy as np
import pytest

import matgen as mg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10

MATS = [
    ("chain_5000", lambda: mg.chain(5000, a=0.5, diag=1.0)),
    ("thin_tail_20k", lambda: mg.thin_tail(20_000, seed=3100)),
    ("stencil3d_14", lambda: mg.stencil3d(14, seed=3)),
    ("stencil2d_48", lambda: mg.stencil2d(48)),
    ("random_400", lambda: mg.random_lower(400, seed=12, density=0.02)),
    ("banded_20k", lambda: mg.banded(20_000, seed=13, band=300, per_row=6)),
]
CFGS = [
    ("plain_sf_t32", dict(select_mode=0, solve_mode=2, tail_rows=32)),
    ("plain_sf_t256", dict(select_mode=0, solve_mode=2, tail_rows=256)),
    ("d2_barrier_t64", dict(select_mode=3, depth=2, solve_mode=1, cta_run_rows=-1,
                            tail_rows=64)),
    ("thin32_sf_t256", dict(select_mode=1, thin_rows=32, max_depth=16, flop_budget=4.0,
                            solve_mode=2, tail_rows=256)),
]


@pytest.mark.parametrize("op", [0, 1], ids=["lower", "upper"])
@pytest.mark.parametrize("cname,kw", CFGS, ids=[c[0] for c in CFGS])
@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_tail_matches_oracle(name, make, cname, kw, op):
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = make() if op == 0 else mg.transposed(make())
    P = B.Plan(A.n, A.row_ptr, A.col, A.val, op=op)
    P.transform(**kw)
    info = P.info()
    if name == "chain_5000":   # every level one row: the whole solve is the tail
        assert info["tail_levels"] == info["nlev_new"]
    b = mg.rhs_uniform(A.n, nrhs=2, seed=21)
    ref = oracle.solve_op(A, b, op)
    bt = torch.as_tensor(b, device="cuda")
    x1 = P.solve(bt[:, 0].contiguous())      # one column: the tail path
    P.check()
    assert oracle.relerr(x1.cpu().numpy(), ref[:, 0]) <= TOL64, (name, cname, info["tail_levels"])
    x = P.solve(bt)                          # two columns: the main kernel alone
    P.check()
    assert oracle.relerr(x.cpu().numpy(), ref) <= TOL64
    x1b = P.solve(bt[:, 1].contiguous())     # repeated solves reuse the records
    P.check()
    assert oracle.relerr(x1b.cpu().numpy(), ref[:, 1]) <= TOL64
    P.close()


def test_tail_on_the_full_thin_tail_matrix():
    """n = 1M: a tail of ~50k positions, so in-tail terms beyond the 16k
    shared-memory window are read from x; also the whole matrix as the tail
    (every level at most 256 rows)."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(1_000_000, seed=3000)
    b = mg.rhs_uniform(A.n, seed=3001)
    ref = oracle.forward_subst(A, b)
    bt = torch.as_tensor(b, device="cuda")
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    for kw in (dict(select_mode=1, thin_rows=32, max_depth=16, flop_budget=4.0, solve_mode=2,
                    tail_rows=32),
               dict(select_mode=0, solve_mode=2, tail_rows=256),
               dict(select_mode=3, depth=3, solve_mode=2, tail_rows=128)):
        P.transform(**kw)
        info = P.info()
        assert info["tail_levels"] > 0, kw
        x = P.solve(bt)
        P.check()
        assert oracle.relerr(x.cpu().numpy(), ref) <= TOL64, (kw, info["tail_levels"])
    P.close()


def test_tail_is_off_where_it_cannot_apply():
    """FP32 + refinement, a negative tail_rows and a tail shorter than 8
    levels leave the main kernel alone; results stay exact."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(40)
    b = mg.rhs_uniform(A.n, seed=5)
    ref = oracle.forward_subst(A, b)
    bt = torch.as_tensor(b, device="cuda")
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    for kw, expect in ((dict(select_mode=0, solve_mode=2, tail_rows=32, precision=1), 0),
                       (dict(select_mode=0, solve_mode=2, tail_rows=-1), 0),
                       (dict(select_mode=0, solve_mode=2, tail_rows=2), 0),
                       (dict(select_mode=0, solve_mode=2, tail_rows=32), None)):
        P.transform(**kw)
        info = P.info()
        if expect is not None:
            assert info["tail_levels"] == expect, kw
        else:
            assert info["tail_levels"] >= 8
        x = P.solve(bt)
        P.check()
        assert oracle.relerr(x.cpu().numpy(), ref) <= TOL64, kw
    P.close()


def test_autotuner_considers_the_tail():
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(100_000, seed=3200)
    b = mg.rhs_uniform(A.n, seed=6)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(select_mode=1, thin_rows=32, max_depth=16, flop_budget=4.0)
    info = P.info()
    assert info["tail_rows"] in (0, 32, 64, 128, 256)
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= TOL64
    P.close()


def test_injected_wait_in_the_tail_times_out():
    """The failure-detection hook on a row that the single-CTA tail would
    solve: the tail (which does not wait) is switched off for good, so the
    bounded wait of the main kernel reports TIMEOUT.  A transform after the
    injection rebuilds the structure from the matrix (the injected
    dependency is gone: the solve is right again) and keeps the tail off."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(20_000, seed=3100)
    kw = dict(select_mode=0, solve_mode=2, tail_rows=32, wait_timeout_ms=200)
    b = mg.rhs_uniform(A.n, seed=4)
    bt = torch.as_tensor(b, device="cuda")
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(**kw)
    assert P.info()["tail_levels"] > 0
    B.sptrsv_debug_inject_wait(P.handle, A.n - 3)
    assert P.info()["tail_levels"] == 0
    P.solve(bt)
    assert B.sptrsv_check(P.handle, 0) == 8   # SPTRSV_ERR_TIMEOUT
    P.close()
    Q = B.Plan(A.n, A.row_ptr, A.col, A.val)
    Q.transform(**kw)
    B.sptrsv_debug_inject_wait(Q.handle, A.n - 3)
    Q.transform(**kw)
    assert Q.info()["tail_levels"] == 0
    x = Q.solve(bt)
    Q.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= TOL64
    Q.close()

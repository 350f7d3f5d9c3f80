"""GPU parity of the generated kernels for thin tail segments (transform
parameter codegen_rows): one thread runs a segment's rows in solve order with
the coefficients, row ids and unknown slots compiled in as constants.  Every
case is compared with the oracle's substitution for its operator; the cases
span a whole-matrix chain, a chain segment after a banded one (its terms on
the banded rows folded beforehand), rewritten chains (b terms folded), the
mirrored operators, rows kept undivided by their diagonal (the generated
division), repeated solves, and the cases where no kernel is generated."""
import numpy as np
import pytest

import matgen as mg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def solve_and_check(A, kw, op=0, nsolves=2, expect_gen=None):
    import torch
    from paper_2103_11445_gb300 import binding as B
    P = B.Plan(A.n, A.row_ptr, A.col, A.val, op=op)
    P.transform(**kw)
    info = P.info()
    if expect_gen is not None:
        ok = expect_gen(info["codegen_segments"]) if callable(expect_gen) else \
            info["codegen_segments"] == expect_gen
        assert ok, info
    for seed in range(nsolves):
        b = mg.rhs_uniform(A.n, seed=70 + seed)
        x = P.solve(torch.as_tensor(b, device="cuda"))
        P.check()
        ref = oracle.solve_op(A, b[:, None], op)[:, 0]
        assert oracle.relerr(x.cpu().numpy(), ref) <= TOL64
    return info


CG = dict(select_mode=0, solve_mode=2, tail_rows=32, codegen_rows=4096)


@pytest.mark.parametrize("op", [0, 1], ids=["lower", "upper"])
def test_whole_matrix_chain(op):
    A = mg.chain(2000, a=0.5, diag=1.0)
    if op == 1:
        A = mg.transposed(A)
    info = solve_and_check(A, CG, op=op, expect_gen=1)
    assert info["tail_levels"] == info["nlev_new"] == 2000
    assert info["codegen_ms"] > 0


def test_chain_with_random_earlier_terms():
    # every row reads the one before and three random earlier ones (mostly
    # more than 32 rows back: shared memory, not registers)
    A = mg.thin_tail(2000, seed=5, chain_frac=1.0)
    solve_and_check(A, CG, expect_gen=1)


@pytest.mark.parametrize("op", [0, 1], ids=["lower", "upper"])
def test_chain_segment_after_banded_levels(op):
    A = mg.thin_tail(20_000, seed=3100)
    if op == 1:
        A = mg.transposed(A)
    kw = dict(CG, tail_rows=256)
    info = solve_and_check(A, kw, op=op)
    if op == 0:   # banded levels stay with the record-driven kernel
        assert info["codegen_segments"] == 1


def test_rewritten_chain_b_terms_folded():
    A = mg.thin_tail(2000, seed=9, chain_frac=1.0)
    # rewritten rows carry more than 16 in-segment terms: the tail is cut
    # into many segments, each with its own generated kernel
    kw = dict(CG, select_mode=1, thin_rows=32, max_depth=8, flop_budget=4.0)
    info = solve_and_check(A, kw, expect_gen=lambda g: g >= 1)
    assert info["rows_rewritten"] > 0


def test_rows_not_divided_by_their_diagonal():
    # rows with L_ii = 2^600 and a neighbour coefficient 2^-500: the quotient
    # underflows, so those rows keep their coefficients and the generated
    # code divides
    n = 2000
    rng = np.random.default_rng(4)
    big = rng.random(n) < 0.3
    diag = np.where(big, 2.0 ** 600, 1.0 + rng.random(n))
    cols = [np.zeros(0, np.int64)] + [np.array([i - 1], np.int64) for i in range(1, n)]
    vals = [np.zeros(0)] + [np.array([2.0 ** -500 if big[i] else 0.5]) for i in range(1, n)]
    A = mg._from_row_lists(n, cols, vals, diag)
    solve_and_check(A, CG, expect_gen=1)


def test_no_kernel_when_not_asked_or_not_thin():
    A = mg.chain(2000, a=0.5, diag=1.0)
    solve_and_check(A, dict(CG, codegen_rows=0), expect_gen=0)
    solve_and_check(A, dict(CG, codegen_rows=1000), expect_gen=0)   # segment too long
    S = mg.stencil2d(48)
    solve_and_check(S, dict(CG, tail_rows=256), expect_gen=0)        # wide levels


def test_generated_and_record_driven_agree_closely():
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(2000, seed=12, chain_frac=1.0)
    b = torch.as_tensor(mg.rhs_uniform(A.n, seed=3), device="cuda")
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(**CG)
    assert P.info()["codegen_segments"] == 1
    xg = P.solve(b).cpu().numpy()
    P.transform(**dict(CG, codegen_rows=0))
    assert P.info()["codegen_segments"] == 0
    xr = P.solve(b).cpu().numpy()
    P.check()
    # the same terms in a different order (oldest first against storage order)
    assert oracle.relerr(xg, xr) <= 1e-13


def test_source_holds_the_matrix_as_constants():
    """The generated source carries the segment itself: one assignment per
    row (its folded constant), one FMA per in-segment term with the
    coefficient as a hexadecimal literal, a function per 32 rows, and no
    load of any structure array (the only memory reads are the folded
    constants and earlier unknowns)."""
    import re
    from paper_2103_11445_gb300 import binding as B
    A = mg.chain(200, a=0.5, diag=2.0)     # x_i = (b_i + 0.5 x_{i-1}) / 2
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(**CG)
    assert P.info()["codegen_segments"] == 1
    src = P.codegen_source(0)
    assert src.count("a = s0[") == 200
    fmas = re.findall(r"a = fma\(([^,]+), (v\[\d+\]|xs\[\d+\]), a\);", src)
    assert len(fmas) == 199
    # coefficient -(-0.5) / 2 = 0.25, written exactly
    assert all(float.fromhex(c) == 0.25 for c, _ in fmas)
    assert len(re.findall(r"__device__ __noinline__ void g\d+\(", src)) == (200 + 31) // 32
    assert re.findall(r"x\[(\d+)\] = a;", src) == [str(i) for i in range(200)]
    for name in ("term", "row_id", "ecol", "eval", "nn["):
        assert name not in src
    with pytest.raises(Exception):
        P.codegen_source(1)                 # one segment only

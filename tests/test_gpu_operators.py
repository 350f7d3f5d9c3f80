"""GPU parity of the other triangular operators (sptrsv_analyze_ex): U x = b,
L^T x = b and U^T x = b, each solved by the same analysis, rewriting
(Sec. III) and solve kernels on a mirrored lower triangle, against the
oracle's substitution for that operator (backward substitution for an upper
triangle, forward substitution for a lower one)."""
import numpy as np
import pytest
import scipy.sparse as sp

import matgen as mg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
OPS = [(1, "upper"), (2, "lower_trans"), (3, "upper_trans")]


def operand(L, op):
    """The CSR handed to the library: the lower matrix itself for the L
    operators, its transpose (an upper matrix) for the U operators."""
    return L if op in (0, 2) else mg.transposed(L)


def lower_form_levels(A, op):
    """Levels of the lower triangle op(A) becomes, in A's row numbering,
    computed with scipy (transpose, row/column reversal) and the oracle."""
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))
    M = S if op in (0, 1) else S.T.tocsr()          # op(A) as a matrix
    upper = op in (1, 2)
    if upper:
        M = M[::-1, ::-1].tocsr()
    M.sort_indices()
    lo = mg.CSR(A.n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)
    lv, nl = oracle.levels(lo)
    return (lv[::-1] if upper else lv), nl


MATS = [
    ("stencil2d_48", lambda: mg.stencil2d(48)),
    ("stencil3d_14", lambda: mg.stencil3d(14, seed=3)),
    ("thin_tail_20k", lambda: mg.thin_tail(20_000, seed=3100)),
    ("random_300", lambda: mg.random_lower(300, seed=11, density=0.03)),
]


@pytest.mark.parametrize("op,opname", OPS, ids=[o[1] for o in OPS])
@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_operator_matches_oracle(op, opname, name, make):
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = operand(make(), op)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val, op=op)
    info = P.info()
    lv_ref, nl_ref = lower_form_levels(A, op)
    assert info["op"] == op and info["nlev"] == nl_ref
    lv, lp, pm = (t.cpu().numpy() for t in P.levels())
    assert np.array_equal(lv, lv_ref)
    assert np.array_equal(np.sort(pm), np.arange(A.n))
    assert np.array_equal(lv[pm], np.repeat(np.arange(nl_ref), np.diff(lp)))
    b = mg.rhs_uniform(A.n, nrhs=3, seed=op)
    ref = oracle.solve_op(A, b, op)
    bt = torch.as_tensor(b, device="cuda")
    for kw in (dict(select_mode=0, solve_mode=1), dict(select_mode=0, solve_mode=2),
               dict(select_mode=3, depth=2, solve_mode=1),
               dict(select_mode=3, depth=2, solve_mode=2),
               dict(select_mode=1, solve_mode=1, cta_run_rows=0),
               dict(select_mode=3, depth=3, solve_mode=2, precision=1)):
        P.transform(**kw)
        x = P.solve(bt)
        P.check()
        err = oracle.relerr(x.cpu().numpy(), ref)
        assert err <= TOL64, (kw, err)
        x1 = P.solve(bt[:, 1].contiguous())
        P.check()
        assert oracle.relerr(x1.cpu().numpy(), ref[:, 1]) <= TOL64, kw
    P.close()


@pytest.mark.parametrize("op,opname", OPS, ids=[o[1] for o in OPS])
def test_full_thin_tail_operators(op, opname):
    """The full 1M-row thin-tail matrix in every operator form, rewritten
    (fixed depth 3) and autotuned."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = operand(mg.thin_tail(1_000_000, seed=3000), op)
    b = mg.rhs_uniform(A.n, seed=3001 + op)
    ref = oracle.solve_op(A, b, op)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val, op=op)
    P.transform(select_mode=3, depth=3)
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), ref) <= TOL64
    P.close()


def test_transformed_export_is_in_the_callers_numbering():
    """For U x = b with fixed depth 1 on an upper chain, the exported rows
    follow the backward closed form: row i (even distance from the end)
    keeps its equation, the others depend on x_{i+2} and b_{i+1}."""
    from paper_2103_11445_gb300 import binding as B
    m, a = 64, 0.5
    U = mg.transposed(mg.chain(m, a=a, diag=1.0))   # x_i - a x_{i+1} = b_i
    P = B.Plan(U.n, U.row_ptr, U.col, U.val, op=1)
    P.transform(select_mode=3, depth=1, solve_mode=2)
    t = {k: v.cpu().numpy() for k, v in P.transformed().items()}
    for i in range(m - 1):
        x0, x1 = t["xptr"][i], t["xptr"][i + 1]
        b0, b1 = t["bptr"][i], t["bptr"][i + 1]
        if (m - 1 - i) % 2 == 0:   # kept level of its segment
            assert list(t["xcol"][x0:x1]) == [i + 1] and b1 == b0
        else:                      # substitutes row i+1's equation
            assert list(t["bcol"][b0:b1]) == [i + 1]
            assert t["bw"][b0] == -a
            if i + 2 < m:
                assert list(t["xcol"][x0:x1]) == [i + 2]
                assert t["xval"][x0] == -(a * a)
    b = mg.rhs_uniform(m, seed=4)
    import torch
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.backward_subst(U, b)) <= 1e-15
    P.close()


def test_batch_with_mixed_operators():
    import torch
    from paper_2103_11445_gb300 import binding as B
    specs = mg.batch_specs(12, seed=4700, n_lo=1e3, n_hi=2e4)
    plans, mats, ops = [], [], []
    for k, spec in enumerate(specs):
        op = k % 4
        A = operand(mg.make_from_spec(spec), op)
        P = B.Plan(A.n, A.row_ptr, A.col, A.val, op=op)
        P.transform(select_mode=3, depth=2, solve_mode=2, precision=1)
        plans.append(P)
        mats.append(A)
        ops.append(op)
    h = B.sptrsv_batch_create([P.handle for P in plans])
    stream = torch.cuda.Stream()
    bs, xs, bnp = [], [], []
    for A, spec in zip(mats, specs):
        b = mg.rhs_uniform(A.n, nrhs=spec["nrhs"], seed=spec["index"]).reshape(A.n, spec["nrhs"])
        bnp.append(b)
        bs.append(torch.as_tensor(b, device="cuda"))
        xs.append(torch.full_like(bs[-1], float("nan")))
    with torch.cuda.stream(stream):
        B.sptrsv_batch_solve(h, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                             [s["nrhs"] for s in specs], stream.cuda_stream)
    assert B.sptrsv_batch_check(h, stream.cuda_stream) == 0
    assert all(B.sptrsv_batch_get_info(h, len(specs))["converged"])
    for A, op, x, b in zip(mats, ops, xs, bnp):
        assert oracle.relerr(x.cpu().numpy(), oracle.solve_op(A, b, op)) <= TOL64, (A.n, op)
    B.sptrsv_batch_destroy(h)
    for P in plans:
        P.close()


def test_wrong_triangle_and_bad_op_are_rejected():
    from paper_2103_11445_gb300 import binding as B
    L = mg.stencil2d(8)
    with pytest.raises(B.SptrsvError) as ei:
        B.Plan(L.n, L.row_ptr, L.col, L.val, op=1)      # a lower matrix is not upper
    assert ei.value.code == 2
    U = mg.transposed(L)
    with pytest.raises(B.SptrsvError) as ei:
        B.Plan(U.n, U.row_ptr, U.col, U.val, op=2)      # L^T needs a lower L
    assert ei.value.code == 2
    with pytest.raises(B.SptrsvError) as ei:
        B.Plan(L.n, L.row_ptr, L.col, L.val, op=7)
    assert ei.value.code == 1


def test_upper_operator_with_column_hint():
    """U x = b with a structure laid out for 8 columns, solved with 5."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    L = mg.thin_tail(8000, seed=91)
    U = mg.transposed(L)
    P = B.Plan(U.n, U.row_ptr, U.col, U.val, op=1)
    P.transform(select_mode=3, depth=2, solve_mode=2, nrhs_hint=8)
    assert P.info()["lanes_per_row"] == 8
    b = mg.rhs_uniform(U.n, nrhs=5, seed=92)
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.solve_op(U, b, 1)) <= TOL64
    P.close()

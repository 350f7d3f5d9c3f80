"""The no-allocation FP32 + FP64-refinement solve (sptrsv_solve_ir_noalloc).

Callers that cannot allocate device memory when they solve (graph capture,
memory fixed by their own pool) use this entry point; it takes its scratch
from a fixed array inside the library.  Here it must give what the regular
sptrsv_solve gives on the same plan, call after call, and refuse sizes
beyond its array.  The file sorts last so that a stop-at-first-failure run
has already run every other test."""
import numpy as np
import pytest

import matgen as mg
import oracle
from gpu_util import plan_for

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
MAX_ELEMS = 1 << 20


@pytest.mark.parametrize("mode", [1, 2], ids=["barrier", "syncfree"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_regular_solve_twice(mode, nrhs):
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(50_000, seed=31)
    P = plan_for(A, select_mode=3, depth=2, solve_mode=mode, precision=1)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        b_np = mg.rhs_uniform(A.n, nrhs=nrhs, seed=100 + call)
        b = torch.as_tensor(b_np, device="cuda")
        x_ref = P.solve(b)
        P.check()
        x = torch.full_like(b, float("nan"))
        B.sptrsv_solve_ir_noalloc(P.handle, b.data_ptr(), x.data_ptr(), nrhs, stream)
        P.check()
        x_np, ref_np = x.cpu().numpy(), x_ref.cpu().numpy()
        assert oracle.relerr(x_np, ref_np) <= TOL64, call
        assert oracle.relerr(x_np, oracle.forward_subst(A, b_np)) <= TOL64, call
    P.close()


def test_noalloc_rejects_oversize_and_wrong_precision():
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(64)
    P = plan_for(A, select_mode=0, solve_mode=1, precision=0)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(B.SptrsvError) as ei:
        B.sptrsv_solve_ir_noalloc(P.handle, b.data_ptr(), x.data_ptr(), 1, 0)
    assert ei.value.code == 9  # BAD_STATE: not an FP32_IR plan
    P.transform(select_mode=0, solve_mode=1, precision=1)
    nrhs = MAX_ELEMS // A.n + 1
    bb = torch.ones(A.n, nrhs, dtype=torch.float64, device="cuda")
    xx = torch.empty_like(bb)
    with pytest.raises(B.SptrsvError) as ei:
        B.sptrsv_solve_ir_noalloc(P.handle, bb.data_ptr(), xx.data_ptr(), nrhs, 0)
    assert ei.value.code == 10  # UNSUPPORTED: beyond the fixed scratch
    # the largest accepted size still solves
    nrhs = MAX_ELEMS // A.n
    b_np = mg.rhs_uniform(A.n, nrhs=nrhs, seed=5)
    bb = torch.as_tensor(b_np, device="cuda")
    xx = torch.empty_like(bb)
    B.sptrsv_solve_ir_noalloc(P.handle, bb.data_ptr(), xx.data_ptr(), nrhs, 0)
    P.check()
    assert oracle.relerr(xx.cpu().numpy(), oracle.forward_subst(A, b_np)) <= TOL64
    P.close()


def test_noalloc_on_a_transposed_operator():
    """L^T x = b through the no-allocation solve: the refinement's residual
    runs on the mirrored triangle with the mirrored index map."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    L = mg.thin_tail(8000, seed=91)
    Q = B.Plan(L.n, L.row_ptr, L.col, L.val, op=B.OP_LOWER_TRANS)
    Q.transform(select_mode=1, solve_mode=2, precision=1)
    b1 = mg.rhs_uniform(L.n, nrhs=2, seed=93)
    bt = torch.as_tensor(b1, device="cuda")
    xt = torch.empty_like(bt)
    B.sptrsv_solve_ir_noalloc(Q.handle, bt.data_ptr(), xt.data_ptr(), 2, 0)
    Q.check()
    assert oracle.relerr(xt.cpu().numpy(), oracle.solve_op(L, b1, oracle.OP_LOWER_TRANS)) <= TOL64
    Q.close()

"""GPU parity of the batched persistent solve (many uneven matrices, 1-32
right-hand sides each, one launch, CUDA-graph replay) against the oracle."""
import numpy as np
import pytest

import matgen as mg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def build(specs, precision, hint=False, **kw):
    import torch
    from paper_2103_11445_gb300 import binding as B
    plans, mats = [], []
    for sp in specs:
        A = mg.make_from_spec(sp)
        P = B.Plan(A.n, A.row_ptr, A.col, A.val)
        if hint:
            kw = dict(kw, nrhs_hint=sp["nrhs"])
        P.transform(precision=precision, **kw)
        plans.append(P)
        mats.append(A)
    return plans, mats


def run_batch(plans, mats, specs, seed, stream):
    import torch
    from paper_2103_11445_gb300 import binding as B
    bs, xs, bnp = [], [], []
    for A, sp in zip(mats, specs):
        b = mg.rhs_uniform(A.n, nrhs=sp["nrhs"], seed=seed + sp["index"])
        b = b.reshape(A.n, sp["nrhs"])
        bnp.append(b)
        bs.append(torch.as_tensor(b, device="cuda"))
        xs.append(torch.full_like(bs[-1], float("nan")))
    return bs, xs, bnp


@pytest.mark.parametrize("precision", [1, 0], ids=["fp32_ir", "fp64"])
def test_batch_matches_oracle_and_replays(precision):
    import torch
    from paper_2103_11445_gb300 import binding as B
    specs = mg.batch_specs(40, seed=4100, n_lo=1e3, n_hi=3e4)
    plans, mats = build(specs, precision, select_mode=1, solve_mode=2)
    h = B.sptrsv_batch_create([P.handle for P in plans])
    stream = torch.cuda.Stream()
    for call in range(2):
        bs, xs, bnp = run_batch(plans, mats, specs, 700 + 31 * call, stream)
        with torch.cuda.stream(stream):
            B.sptrsv_batch_solve(h, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                                 [sp["nrhs"] for sp in specs], stream.cuda_stream)
        assert B.sptrsv_batch_check(h, stream.cuda_stream) == 0
        info = B.sptrsv_batch_get_info(h, len(specs))
        for A, x, b in zip(mats, xs, bnp):
            err = oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b))
            assert err <= TOL64, (call, A.n, err)
        if precision == 1:
            assert all(info["converged"])
        assert min(info["cta_count"]) >= 1
        assert info["graph"] == 1
    B.sptrsv_batch_destroy(h)
    for P in plans:
        P.close()


def test_batch_on_default_stream_runs_without_graph():
    import torch
    from paper_2103_11445_gb300 import binding as B
    specs = mg.batch_specs(6, seed=4200, n_lo=1e3, n_hi=1e4)
    plans, mats = build(specs, 1, select_mode=0, solve_mode=2)
    h = B.sptrsv_batch_create([P.handle for P in plans])
    bs, xs, bnp = run_batch(plans, mats, specs, 5, None)
    B.sptrsv_batch_solve(h, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                         [sp["nrhs"] for sp in specs], 0)
    assert B.sptrsv_batch_check(h, 0) == 0
    assert B.sptrsv_batch_get_info(h, len(specs))["graph"] == 0
    for A, x, b in zip(mats, xs, bnp):
        assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= TOL64
    B.sptrsv_batch_destroy(h)


def test_batch_rejects_mixed_precision():
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(16)
    P1 = B.Plan(A.n, A.row_ptr, A.col, A.val).transform(precision=1)
    P2 = B.Plan(A.n, A.row_ptr, A.col, A.val).transform(precision=0)
    with pytest.raises(B.SptrsvError) as ei:
        B.sptrsv_batch_create([P1.handle, P2.handle])
    assert ei.value.code == 1


def test_batch_256_uneven_matrices():
    """The mixture of 256 matrices (n log-uniform in [1e3, 2e5], 5-point,
    7-point and random-banded, 1-32 right-hand sides each), FP32 values with
    FP64 refinement, one graph-replayed launch; two columns of every matrix
    are checked against the oracle."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    specs = mg.batch_specs(256, seed=4000)
    plans, mats = build(specs, 1, hint=True, select_mode=1, solve_mode=2)
    h = B.sptrsv_batch_create([P.handle for P in plans])
    stream = torch.cuda.Stream()
    bs, xs, bnp = run_batch(plans, mats, specs, 9, stream)
    with torch.cuda.stream(stream):
        B.sptrsv_batch_solve(h, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                             [sp["nrhs"] for sp in specs], stream.cuda_stream)
    assert B.sptrsv_batch_check(h, stream.cuda_stream) == 0
    info = B.sptrsv_batch_get_info(h, len(specs))
    assert all(info["converged"]) and info["graph"] == 1
    for A, x, b, sp in zip(mats, xs, bnp, specs):
        cols = sorted({0, sp["nrhs"] - 1})
        ref = oracle.forward_subst(A, np.ascontiguousarray(b[:, cols]))
        err = oracle.relerr(x.cpu().numpy()[:, cols], ref)
        assert err <= TOL64, (sp, err)
    B.sptrsv_batch_destroy(h)


def test_batch_groups_are_timed_and_resized():
    """Every group's time of the last solve is reported; the first solve
    re-sizes the groups from measured times (every matrix keeps at least one
    CTA, the table never holds more CTAs than the grid), and the solves stay
    right after the re-sizing."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    mats = [mg.stencil3d(12, seed=1), mg.chain(3000, a=0.5, diag=1.0),
            mg.thin_tail(20_000, seed=4), mg.stencil2d(30)]
    plans = []
    for A in mats:
        P = B.Plan(A.n, A.row_ptr, A.col, A.val)
        P.transform(select_mode=1, solve_mode=2, precision=1)
        plans.append(P)
    h = B.sptrsv_batch_create([P.handle for P in plans])
    with pytest.raises(B.SptrsvError):
        B.sptrsv_batch_get_times(h, len(mats))
    bs = [torch.as_tensor(mg.rhs_uniform(A.n, seed=i), device="cuda") for i, A in enumerate(mats)]
    xs = [torch.empty_like(b) for b in bs]
    s = torch.cuda.Stream()
    for _ in range(3):
        B.sptrsv_batch_solve(h, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                             [1] * len(mats), s.cuda_stream)
        s.synchronize()
        assert B.sptrsv_batch_check(h, s.cuda_stream) == 0
        for A, b, x in zip(mats, bs, xs):
            assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b.cpu().numpy())) <= 1e-10
    ms = B.sptrsv_batch_get_times(h, len(mats))
    assert all(t > 0 for t in ms)
    info = B.sptrsv_batch_get_info(h, len(mats))
    assert min(info["cta_count"]) >= 1
    # the chain (3000 levels of one row) is the slowest and got the most time
    assert max(ms) == ms[1]
    B.sptrsv_batch_destroy(h)
    for P in plans:
        P.close()

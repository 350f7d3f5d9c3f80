"""GPU checks of the per-segment selection (SELECT_SEGMODEL) with the shipped
network: the library's segmentation is the minimum-sum segmentation of the
oracle (oracle.critpath.select_min_sum) over the costs 2^prediction of the
library's own segment features, and the transformed solve matches the
oracle's substitution; the level times it is trained on add up to the solve
and every new level gets one."""
import os

import numpy as np
import pytest

import matgen as mg
import oracle
from oracle import critpath as cpo

pytestmark = pytest.mark.gpu

CASES = [
    ("stencil2d_120", lambda: mg.stencil2d(120)),
    ("stencil3d_30", lambda: mg.stencil3d(30, seed=7)),
    ("thin_tail_30k", lambda: mg.thin_tail(30_000, seed=8)),
    ("banded_20k", lambda: mg.banded(20_000, seed=9, band=300, per_row=6)),
]
LAUNCH = dict(solve_mode=2, lanes_per_row=2, block_threads=128, grid_blocks=0, tail_rows=-1,
              cta_run_rows=-1)


@pytest.fixture(scope="module")
def net():
    from paper_2103_11445_gb300 import binding as B
    from paper_2103_11445_gb300 import costmodel as cm
    if not os.path.exists(cm.SEG_WEIGHTS_BIN):
        pytest.skip("no shipped segment network")
    m = cm.CostModel.load(cm.SEG_WEIGHTS_BIN)
    B.sptrsv_segmodel_set_default(m.handle)
    yield m
    B.sptrsv_segmodel_set_default(0)
    m.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_segmentation_is_the_min_sum_of_predicted_costs(net, name, make):
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = make()
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(select_mode=B.SELECT_SEGMODEL, max_depth=4, **LAUNCH)
    first, depth = P.segments()
    feat, ok = P.segment_features(4)
    nlev = feat.shape[0]
    pred = np.zeros((nlev, 5), np.float32)
    pred[ok] = net.predict(feat[ok])
    cost = np.exp2(pred.astype(np.float64))
    assert list(zip(first, depth)) == cpo.select_min_sum(cost, ok)
    b = mg.rhs_uniform(A.n, seed=1)
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= 1e-10


def test_level_times_add_up_to_the_solve():
    import torch
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil3d(40, seed=3)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(select_mode=B.SELECT_FIXED, depth=1, **LAUNCH)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    us = P.level_times(b, reps=3)
    assert us.shape == (P.info()["nlev_new"],) and (us >= 0).all()
    total = float(us.sum())
    t = []
    x = torch.empty_like(b)
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        P.solve(b, x)
        e1.record()
        e1.synchronize()
        t.append(e0.elapsed_time(e1) * 1e3)
    P.check()
    # the stamps cover the solve after its start-up, within the launch
    assert 0.3 * np.median(t) <= total <= 1.2 * np.median(t), (total, t)
    with pytest.raises(Exception):          # the tail or several columns: not stamped
        P.transform(select_mode=B.SELECT_FIXED, depth=1, **dict(LAUNCH, stage_z=-1))
        P.level_times(b)

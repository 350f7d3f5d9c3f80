"""What the trained cost model gains over the method without it.

On matrices drawn with a seed the network never saw, the depth it picks
(SELECT_COSTMODEL, shipped weights) must solve correctly and be faster than
the thin-level heuristic H (the selection without the network) and than the
plain level sets, measured live on the GPU."""
import os

import numpy as np
import pytest

import matgen as mg
import oracle

pytestmark = pytest.mark.gpu


def test_trained_network_beats_the_heuristic():
    import torch
    from paper_2103_11445_gb300 import binding as B
    from paper_2103_11445_gb300 import costmodel as cm
    if not os.path.exists(cm.WEIGHTS):
        pytest.skip("no trained weights shipped")
    net = cm.CostModel.load()
    specs = mg.batch_specs(12, seed=9000, n_lo=2e4, n_hi=1.5e5, nrhs_max=1,
                           band_range=(5, 20))
    t_cm, t_h, t_plain, picks = [], [], [], []
    for sp in specs:
        A = mg.make_from_spec(sp)
        P = B.Plan(A.n, A.row_ptr, A.col, A.val)
        net.attach(P)
        P.transform(select_mode=B.SELECT_COSTMODEL, solve_mode=B.SOLVE_SYNCFREE)
        picks.append(P.info()["chosen_depth"])
        b = mg.rhs_uniform(A.n, seed=sp["seed"])
        x = P.solve(torch.as_tensor(b, device="cuda"))
        P.check()
        assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= 1e-10
        t_cm.append(cm.label_time(P, A.n, reps=7, select_mode=B.SELECT_COSTMODEL))
        t_h.append(cm.heuristic_time(P, A.n, reps=7))
        t_plain.append(cm.label_time(P, A.n, reps=7, select_mode=B.SELECT_NONE))
        P.close()
    net.close()
    geo = lambda a, b: float(np.exp(np.mean(np.log(np.asarray(a) / np.asarray(b)))))
    vs_h, vs_plain = geo(t_h, t_cm), geo(t_plain, t_cm)
    print(f"picks {picks}; geo-mean speed-up vs heuristic {vs_h:.3f}, vs plain {vs_plain:.3f}")
    assert all(p in cm.CANDIDATES for p in picks)
    assert vs_h > 1.15
    assert vs_plain > 1.10

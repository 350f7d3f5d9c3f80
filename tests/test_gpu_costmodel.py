"""GPU parity of the cost-model network (forward, gradients, Adam) against the
FP64 oracle, of the candidate features against the oracle transform, and the
selection plumbing of SELECT_COSTMODEL."""
import os

import numpy as np
import pytest

import matgen as mg
import oracle
from oracle import mlp as omlp
from oracle import rewrite as rw
from gpu_util import assert_close_to_oracle, gpu_solve, plan_for

pytestmark = pytest.mark.gpu

F, H = 17, 64


def oracle_params(flat, n_in=F, hidden=H):
    o = 0
    out = {}
    for name, shape in (("W1", (n_in, hidden)), ("b1", (hidden,)), ("W2", (hidden, hidden)),
                        ("b2", (hidden,)), ("W3", (hidden, 1)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = flat[o:o + size].astype(np.float64).reshape(shape)
        o += size
    return out


def flat_of(p):
    return np.concatenate([p[k].ravel() for k in omlp.PARAM_NAMES])


def setup_net(seed=0, N=300):
    import torch
    from paper_2103_11445_gb300 import costmodel as cm
    rng = np.random.default_rng(seed)
    params = cm.init_params(F, H, seed)
    params[F * H:F * H + H] = rng.uniform(-0.2, 0.2, H)  # non-zero biases
    X = rng.standard_normal((N, F)).astype(np.float32)
    t = rng.standard_normal(N).astype(np.float32)
    net = cm.CostModel(params)
    return net, params, X, t


def test_forward_matches_oracle():
    net, params, X, _ = setup_net()
    y = net.predict(X)
    ref, _ = omlp.forward(oracle_params(params), X.astype(np.float64))
    assert np.allclose(y, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    net.close()


def test_gradients_match_oracle():
    import torch
    from paper_2103_11445_gb300 import binding as B
    net, params, X, t = setup_net(1)
    dX = torch.as_tensor(X, device="cuda")
    dt = torch.as_tensor(t, device="cuda")
    g = torch.empty(params.size, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    B.sptrsv_mlp_grads(net.handle, dX.data_ptr(), dt.data_ptr(), X.shape[0], g.data_ptr(),
                       loss.data_ptr(), 0)
    torch.cuda.synchronize()
    ref_loss, ref_g = omlp.loss_and_grads(oracle_params(params), X.astype(np.float64),
                                          t.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    ref = flat_of(ref_g)
    got = g.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref).max() + 1e-7)
    net.close()


def test_adam_step_matches_oracle():
    import torch
    from paper_2103_11445_gb300 import binding as B
    net, params, X, t = setup_net(2)
    dX = torch.as_tensor(X, device="cuda")
    dt = torch.as_tensor(t, device="cuda")
    lr = 1e-3
    B.sptrsv_mlp_train_step(net.handle, dX.data_ptr(), dt.data_ptr(), X.shape[0], lr, 0, 0)
    torch.cuda.synchronize()
    p = oracle_params(params)
    _, g = omlp.loss_and_grads(p, X.astype(np.float64), t.astype(np.float64))
    st = omlp.adam_init(p)
    omlp.adam_step(p, g, st, lr=lr)
    ref = flat_of(p)
    got = net.params()
    gref = np.abs(flat_of(g))
    firm = gref > 1e-5 * gref.max()      # Adam's first step is ~lr * sign(g)
    assert np.all(np.abs(got - ref)[firm] <= 1e-6)
    net.close()


def test_training_fits_a_smooth_target():
    from paper_2103_11445_gb300 import costmodel as cm
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2000, F)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.3 * X[:, 12]).astype(np.float32)
    net = cm.CostModel(seed=4)
    hist = net.fit(X, y, epochs=600, lr=3e-3, log_every=100)
    assert hist[-1][1] < 0.05 * hist[0][1]
    net.close()


@pytest.mark.parametrize("code", [0, 1, 3, 8, 108, 116])
def test_features_match_oracle_transform(code):
    from paper_2103_11445_gb300 import binding as B
    A = mg.thin_tail(20_000, seed=3000)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    f = B.sptrsv_costmodel_features(P.handle, [code])[0]
    lv, nl = oracle.levels(A)
    thin = code >= 100
    d = code - 100 if thin else code
    if d:
        tau, rho = (32, 4.0) if thin else (10**12, float("inf"))
        tr = rw.transform(A, lv, nl, tau=tau, d_max=d, rho=rho, max_fill=1024)
        nnew, added, rewritten = tr.nlev_new, tr.added_flops, len(tr.rows)
    else:
        nnew, added, rewritten = nl, 0, 0
    sizes = np.bincount(lv)
    offd = np.diff(A.row_ptr) - 1
    assert np.isclose(f[0], np.log2(A.n), rtol=1e-6) and np.isclose(f[3], np.log2(nl), rtol=1e-6)
    assert f[12] == d and f[16] == (1.0 if thin else 0.0)
    assert np.isclose(f[13], np.log2(nnew), rtol=1e-6)
    assert np.isclose(f[14], (rw.total_flops(A) + added) / rw.total_flops(A), rtol=1e-6)
    assert np.isclose(f[15], rewritten / A.n, rtol=1e-6)
    assert np.isclose(f[5], (sizes < 32).mean(), rtol=1e-6)
    hist = [(offd == 0).mean(), ((offd >= 1) & (offd <= 2)).mean(),
            ((offd >= 3) & (offd <= 6)).mean(), (offd >= 7).mean()]
    assert np.allclose(f[8:12], hist, rtol=1e-6)
    P.close()


@pytest.mark.parametrize("sign,expect", [(1.0, 0), (-1.0, 116)])
def test_costmodel_selection_takes_the_argmin(sign, expect):
    """A hand-built network whose output is +d or -d (d = feature 12) must
    make the plan pick the plain level sets (code 0) or the deepest candidate
    (thin levels only, depth 16: code 116); the solve must still match the
    oracle."""
    from paper_2103_11445_gb300 import binding as B
    from paper_2103_11445_gb300 import costmodel as cm
    params = np.zeros(B.sptrsv_mlp_num_params(F, H), np.float32)
    params[12 * H + 0] = 1.0                 # W1[12][0]: hidden unit 0 = relu(d)
    params[F * H + H + 0 * H + 0] = 1.0      # W2[0][0]
    params[F * H + H + H * H + H + 0] = sign  # W3[0]
    net = cm.CostModel(params)               # identity normalisation
    A = mg.stencil2d(32)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    net.attach(P)
    P.transform(select_mode=B.SELECT_COSTMODEL, solve_mode=B.SOLVE_SYNCFREE)
    info = P.info()
    assert info["chosen_depth"] == expect
    if expect:   # stencil2d(32): levels under 32 rows are the 31 + 31 corner levels
        lv, nl = oracle.levels(A)
        tr = rw.transform(A, lv, nl, tau=32, d_max=16, rho=4.0, max_fill=1024)
        assert info["nlev_new"] == tr.nlev_new < info["nlev"]
    b = mg.rhs_uniform(A.n, seed=2)
    import torch
    x = P.solve(torch.as_tensor(b, device="cuda"))
    P.check()
    assert oracle.relerr(x.cpu().numpy(), oracle.forward_subst(A, b)) <= 1e-10
    P.close()
    net.close()


def test_costmodel_fallback_is_the_heuristic():
    from paper_2103_11445_gb300 import binding as B
    A = mg.stencil2d(32)
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    P.transform(select_mode=B.SELECT_COSTMODEL, solve_mode=B.SOLVE_BARRIER)
    seg_cm = P.segments()
    assert P.info()["chosen_depth"] == -1
    P.transform(select_mode=B.SELECT_HEURISTIC, solve_mode=B.SOLVE_BARRIER)
    assert P.segments() == seg_cm
    P.close()


def test_network_file_round_trip_and_default_model(tmp_path):
    """sptrsv_mlp_save / sptrsv_mlp_load and the process-wide model of
    sptrsv_costmodel_load / _save, through the C ABI: the loaded network has
    the same weights and normalisation, predicts the same values, and
    SELECT_COSTMODEL without an attached network picks the same candidate
    as with the original attached."""
    import torch
    from paper_2103_11445_gb300 import binding as B
    from paper_2103_11445_gb300.costmodel import CostModel, N_FEATURES
    rng = np.random.default_rng(5)
    X = rng.normal(size=(64, N_FEATURES)).astype(np.float32) * 3 + 1
    y = rng.normal(size=64).astype(np.float32)
    m = CostModel(seed=3)
    m.fit(X, y, epochs=20)
    f1 = str(tmp_path / "net.bin")
    m.save(f1)
    q = CostModel.load(f1)
    assert np.array_equal(q.params(), m.params())
    assert np.array_equal(q.mean, m.mean) and np.array_equal(q.std, m.std)
    assert np.array_equal(q.predict(X), m.predict(X))
    # the statistics are the library's: column means and deviations of X
    assert np.allclose(m.mean, X.mean(axis=0), rtol=1e-5, atol=1e-5)
    assert np.allclose(m.std, X.std(axis=0), rtol=1e-4)
    # the process-wide model
    A = mg.stencil3d(24, seed=8)
    P = plan_for(A)
    m.attach(P)
    P.transform(select_mode=2, solve_mode=2)
    pick = P.info()["chosen_depth"]
    B.sptrsv_costmodel_load(f1)
    f2 = str(tmp_path / "default.bin")
    B.sptrsv_costmodel_save(f2)
    assert open(f1, "rb").read() == open(f2, "rb").read()
    Q = plan_for(A)
    Q.transform(select_mode=2, solve_mode=2)
    assert Q.info()["chosen_depth"] == pick
    b = mg.rhs_uniform(A.n, seed=1)
    assert_close_to_oracle(A, gpu_solve(Q, b), b, 1e-10)
    B.sptrsv_costmodel_set_default(0)
    Q.transform(select_mode=2, solve_mode=2)
    assert Q.info()["chosen_depth"] == -1        # no network: heuristic H
    with pytest.raises(B.SptrsvError):
        B.sptrsv_costmodel_save(str(tmp_path / "none.bin"))
    for c in (m, q):
        c.close()
    P.close()
    Q.close()

"""Pins of the cost-model network oracle: a forward pass worked by hand,
central finite differences for every gradient, and the closed form of Adam's
first step."""
import numpy as np

from oracle import mlp


def test_forward_by_hand():
    # F=2, H=2; every quantity below is worked out by hand
    p = dict(W1=np.array([[1.0, -1.0], [2.0, 0.5]]), b1=np.array([0.0, 1.0]),
             W2=np.array([[1.0, 0.0], [-1.0, 2.0]]), b2=np.array([-1.0, 0.0]),
             W3=np.array([[3.0], [0.5]]), b3=np.array([0.25]))
    X = np.array([[1.0, 1.0], [-2.0, 0.0]])
    # row 0: z1 = (3, 0.5) h1 = (3, 0.5); z2 = (3-0.5-1, 1) = (1.5, 1); y = 4.5+0.5+0.25
    # row 1: z1 = (-2, 3) h1 = (0, 3); z2 = (-3-1, 6) -> h2 = (0, 6); y = 3 + 0.25
    y, _ = mlp.forward(p, X)
    assert y.tolist() == [5.25, 3.25]
    assert mlp.loss(p, X, np.array([5.0, 3.0])) == (0.25 ** 2 + 0.25 ** 2) / 2


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    F, H, N = 5, 7, 11
    p = mlp.init_params(F, H, seed=3)
    for k in ("b1", "b2"):
        p[k] = rng.uniform(-0.3, 0.3, H)
    X = rng.standard_normal((N, F))
    tgt = rng.standard_normal(N)
    _, g = mlp.loss_and_grads(p, X, tgt)
    h = 1e-6
    for name in mlp.PARAM_NAMES:
        flat = p[name].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, X, tgt)
            flat[idx] = old - h
            lm = mlp.loss(p, X, tgt)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so p1 = p0 - lr*g/(|g|+eps)
    rng = np.random.default_rng(1)
    p = mlp.init_params(4, 6, seed=2)
    g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    p0 = {k: v.copy() for k, v in p.items()}
    st = mlp.adam_init(p)
    mlp.adam_step(p, g, st, lr=0.01)
    for k in p:
        assert np.allclose(p[k], p0[k] - 0.01 * g[k] / (np.abs(g[k]) + 1e-8),
                           rtol=1e-12, atol=1e-15)


def test_training_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((256, 3))
    tgt = X @ np.array([0.5, -1.0, 2.0]) + 0.3
    p = mlp.init_params(3, 16, seed=5)
    st = mlp.adam_init(p)
    l0 = mlp.loss(p, X, tgt)
    for _ in range(300):
        _, g = mlp.loss_and_grads(p, X, tgt)
        mlp.adam_step(p, g, st, lr=0.01)
    assert mlp.loss(p, X, tgt) < 0.05 * l0

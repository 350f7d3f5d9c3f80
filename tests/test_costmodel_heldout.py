"""The shipped cost-model network on the 400 held-out matrices of its data set
(the last fifth by matrix, never trained on): its pick against the fastest of
the nine candidate selections for each matrix (regret), against the thin-level
heuristic H and against the plain level sets.  The labels are the solve times
stored with the data (log2 us, measured on the GPU when the set was
collected); the network is evaluated by the oracle's FP64 forward pass, so
this needs no GPU."""
import os

import numpy as np
import pytest

from oracle import mlp

HERE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2103_11445_gb300")
WEIGHTS = os.path.join(HERE, "costmodel_weights.npz")
DATA = os.path.join(HERE, "costmodel_data.npz")
HELD_OUT_FROM = 1600   # matrices 1600..1999 (training used the first 80 %)


def network(w):
    F, H = int(w["n_in"]), int(w["hidden"])
    flat, o, p = w["params"], 0, {}
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (H, 1)), ("b3", (1,))):
        size = int(np.prod(shape))
        p[name] = flat[o:o + size].astype(np.float64).reshape(shape)
        o += size
    assert o == flat.size
    return p


@pytest.mark.skipif(not (os.path.exists(WEIGHTS) and os.path.exists(DATA)),
                    reason="no shipped network or data set")
def test_held_out_regret():
    w, d = np.load(WEIGHTS), np.load(DATA)
    assert list(w["candidates"]) == list(d["candidates"])
    X, y, g, h = d["X"], d["y"], d["group"], d["h"]
    te = g >= HELD_OUT_FROM
    pred = mlp.forward(network(w), (X[te] - w["mean"]) / w["std"])[0].reshape(-1)
    yt, gt = y[te], g[te]
    pick, best, heur, plain = [], [], [], []
    for k in np.unique(gt):
        s = gt == k
        pick.append(2.0 ** yt[s][np.argmin(pred[s])])
        best.append(2.0 ** yt[s].min())
        heur.append(2.0 ** h[k])
        plain.append(2.0 ** yt[s][0])          # candidate 0: no rewriting
    pick, best, heur, plain = map(np.asarray, (pick, best, heur, plain))
    regret = pick / best
    geo = lambda a: float(np.exp(np.mean(np.log(a))))
    print(f"held out {len(regret)}: mean regret {regret.mean():.4f}, picks the best "
          f"{np.mean(regret <= 1.0001):.3f}, geo speed-up vs H {geo(heur / pick):.3f}, "
          f"vs plain {geo(plain / pick):.3f}")
    assert len(regret) == 400
    assert regret.mean() <= 1.02              # measured 1.003
    assert np.mean(regret <= 1.0001) >= 0.85  # measured 0.90
    assert geo(heur / pick) >= 1.4            # measured 1.51
    assert geo(plain / pick) >= 1.4           # measured 1.55

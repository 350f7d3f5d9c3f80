"""The shipped per-segment network (SELECT_SEGMODEL) against the level times
it was trained on: a stored subsample of the training rows (features of one
new level of one timed segmentation, log2 of the microseconds that level
added to a solve on the GPU).  The network file is read as the library
writes it and evaluated by the oracle's FP64 forward pass, so this needs no
GPU; it pins that the shipped file is the trained network."""
import os
import struct

import numpy as np
import pytest

from oracle import mlp

HERE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2103_11445_gb300")
WEIGHTS = os.path.join(HERE, "segmodel_weights.bin")
DATA = os.path.join(HERE, "segmodel_data.npz")


def read_network(path):
    raw = open(path, "rb").read()
    assert raw[:8] == b"SPTRSVNN"
    version, F, H, has_norm = struct.unpack("<4i", raw[8:24])
    assert version == 1 and has_norm == 1
    npar = F * H + H + H * H + H + H + 1
    flat = np.frombuffer(raw[24:24 + 4 * npar], np.float32)
    mean = np.frombuffer(raw[24 + 4 * npar:24 + 4 * (npar + F)], np.float32)
    std = np.frombuffer(raw[24 + 4 * (npar + F):24 + 4 * (npar + 2 * F)], np.float32)
    assert len(raw) == 24 + 4 * (npar + 2 * F)
    p, o = {}, 0
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (H, 1)), ("b3", (1,))):
        size = int(np.prod(shape))
        p[name] = flat[o:o + size].astype(np.float64).reshape(shape)
        o += size
    return F, p, mean.astype(np.float64), std.astype(np.float64)


@pytest.mark.skipif(not (os.path.exists(WEIGHTS) and os.path.exists(DATA)),
                    reason="no shipped segment network or data")
def test_network_fits_its_stored_level_times():
    F, p, mean, std = read_network(WEIGHTS)
    d = np.load(DATA)
    X, y = d["X"].astype(np.float64), d["y"].astype(np.float64)
    assert F == 8 and X.shape[1] == 8
    # feature sanity: d in 0..4, fractions in [0, 1], rows >= 1
    assert set(np.unique(X[:, 4]).tolist()) <= {0.0, 1.0, 2.0, 3.0, 4.0}
    assert (X[:, 5] >= 0).all() and (X[:, 5] <= 1).all() and (X[:, 0] >= 1).all()
    pred = mlp.forward(p, (X - mean) / std)[0].reshape(-1)
    mse = float(np.mean((pred - y) ** 2))
    # log2 units: the training run ended at 0.361 on all 98,225 rows
    assert mse <= 0.42, mse
    # the network orders levels by cost: its predictions rank-correlate
    # with the measured times
    r = np.corrcoef(np.argsort(np.argsort(pred)), np.argsort(np.argsort(y)))[0, 1]
    assert r >= 0.6, r

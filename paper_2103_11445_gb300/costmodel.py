"""Learned choice of the rewriting depth.

The paper chooses the rows to rewrite by hand (Sec. IV).  Here a small network
(``libsptrsv`` cost-model kernels: 17 features -> 64 -> 64 -> 1, ReLU, FP32,
trained with Adam on the GPU) predicts the log solve time of every candidate
in CANDIDATES -- "merge every d+1 levels" (code d) or "rewrite only the levels
under 32 rows, up to d deep" (code 100 + d) -- and
``SPTRSV_SELECT_COSTMODEL`` keeps the argmin.
Heuristic H remains the fallback when no network is attached, and the
baseline the network is judged against.

Training data come from the solver itself: for every seeded synthetic matrix
(``matgen`` mixtures) and every candidate, the library's features of that
candidate and the measured time of the library's own solve of the rewritten
plan (the faster of two launch shapes, median of a few solves each, L2
flushed before each).

    python -m paper_2103_11445_gb300.costmodel collect --count 600 --out data.npz
    python -m paper_2103_11445_gb300.costmodel train --data data.npz --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

from . import binding as B

CANDIDATES = (0, 1, 2, 3, 4, 6, 8, 108, 116)
THIN_ONLY = 100      # code 100 + d: levels under THIN_ROWS rows only, depth <= d
THIN_ROWS = 32
THIN_BUDGET = 4.0
N_FEATURES = 17
HIDDEN = 64
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.npz")
# the same network in the library's file format (sptrsv_costmodel_load)
WEIGHTS_BIN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.bin")
# Launch shapes of the timing labels: a label is the fastest of these
# (sync-free kernel, 128 threads per CTA): one lane per row on one CTA per
# SM, and four lanes per row on four CTAs per SM -- between them the shapes
# the autotuner ends up with on the matrices measured (deep chains vs wide
# levels), at a fraction of a full autotuning run per candidate.
LABEL_LAUNCHES = (dict(lanes_per_row=1, ctas_per_sm=1), dict(lanes_per_row=4, ctas_per_sm=4))


def init_params(n_in: int = N_FEATURES, hidden: int = HIDDEN, seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, shape)

    parts = [he(n_in, (n_in, hidden)), np.zeros(hidden), he(hidden, (hidden, hidden)),
             np.zeros(hidden), he(hidden, (hidden, 1)), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


class CostModel:
    """A cost-model network living on the current CUDA device.  Feature
    standardisation is the library's (sptrsv_mlp_fit_normalization /
    sptrsv_mlp_normalize): features go to the device as they are."""

    def __init__(self, params: np.ndarray | None = None, mean=None, std=None,
                 n_in: int = N_FEATURES, hidden: int = HIDDEN, seed: int = 0,
                 handle: int = 0):
        self.n_in, self.hidden = n_in, hidden
        if handle:
            self.handle = handle
            return
        if params is None:
            params = init_params(n_in, hidden, seed)
        self.handle = B.sptrsv_mlp_create(n_in, hidden, params)
        if mean is not None and std is not None:
            B.sptrsv_mlp_set_normalization(self.handle, np.asarray(mean, np.float32),
                                           np.asarray(std, np.float32))

    @property
    def mean(self) -> np.ndarray:
        return B.sptrsv_mlp_get_normalization(self.handle, self.n_in)[0]

    @property
    def std(self) -> np.ndarray:
        return B.sptrsv_mlp_get_normalization(self.handle, self.n_in)[1]

    def _normalised(self, X: np.ndarray, fit: bool = False):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        if fit:
            B.sptrsv_mlp_fit_normalization(self.handle, Xd.data_ptr(), Xd.shape[0], stream)
        B.sptrsv_mlp_normalize(self.handle, Xd.data_ptr(), Xd.shape[0], Xd.data_ptr(), stream)
        return Xd

    # -- training ----------------------------------------------------------
    def fit(self, X: np.ndarray, y: np.ndarray, epochs: int = 3000, lr: float = 3e-3,
            log_every: int = 0) -> list:
        """Full-batch Adam on features standardised by the library (statistics
        from X, computed on the device)."""
        import torch
        Xn = self._normalised(X, fit=True)
        t = torch.as_tensor(y, dtype=torch.float32, device=Xn.device)
        loss = torch.zeros(1, dtype=torch.float32, device=Xn.device)
        stream = torch.cuda.current_stream().cuda_stream
        hist = []
        for e in range(epochs):
            B.sptrsv_mlp_train_step(self.handle, Xn.data_ptr(), t.data_ptr(), Xn.shape[0], lr,
                                    loss.data_ptr(), stream)
            if log_every and (e % log_every == 0 or e == epochs - 1):
                hist.append((e, float(loss.item())))
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        import torch
        Xn = self._normalised(X)
        y = torch.empty(Xn.shape[0], dtype=torch.float32, device=Xn.device)
        B.sptrsv_mlp_forward(self.handle, Xn.data_ptr(), Xn.shape[0], y.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        return y.cpu().numpy()

    def params(self) -> np.ndarray:
        return B.sptrsv_mlp_get_params(self.handle, self.n_in, self.hidden)

    # -- persistence ------------------------------------------------------------
    def save(self, path: str = WEIGHTS) -> None:
        """The library's network file (sptrsv_mlp_save) for a path ending in
        .bin, else an .npz archive with the same contents."""
        if path.endswith(".bin"):
            B.sptrsv_mlp_save(self.handle, path)
            return
        np.savez(path, params=self.params(), mean=self.mean, std=self.std,
                 n_in=self.n_in, hidden=self.hidden, candidates=np.array(CANDIDATES))

    @classmethod
    def load(cls, path: str = WEIGHTS) -> "CostModel":
        if path.endswith(".bin"):
            import struct
            with open(path, "rb") as fh:
                _, n_in, hidden, _ = struct.unpack("<4i", fh.read(24)[8:])
            return cls(n_in=n_in, hidden=hidden, handle=B.sptrsv_mlp_load(path))
        d = np.load(path)
        return cls(d["params"], d["mean"], d["std"], int(d["n_in"]), int(d["hidden"]))

    def attach(self, plan: "B.Plan") -> None:
        B.sptrsv_set_costmodel(plan.handle, self.handle)

    def close(self) -> None:
        if self.handle:
            B.sptrsv_mlp_destroy(self.handle)
            self.handle = 0


# --- data ------------------------------------------------------------------------

def time_solves(plan: "B.Plan", n: int, reps: int = 5) -> float:
    """Median solve time in microseconds, L2 flushed before each solve."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    b = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    plan.solve(b, x)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.solve(b, x)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    plan.check()
    return statistics.median(ts)


def label_time(plan: "B.Plan", n: int, reps: int = 3, **select) -> float:
    """The label of a selection: its fastest solve over LABEL_LAUNCHES (us)."""
    sms = plan.info()["num_sms"]
    best = float("inf")
    for lk in LABEL_LAUNCHES:
        plan.transform(**select, solve_mode=B.SOLVE_SYNCFREE, block_threads=128,
                       lanes_per_row=lk["lanes_per_row"], grid_blocks=lk["ctas_per_sm"] * sms)
        best = min(best, time_solves(plan, n, reps))
    return best


def heuristic_time(plan: "B.Plan", n: int, reps: int = 3) -> float:
    return label_time(plan, n, reps, select_mode=B.SELECT_HEURISTIC)


def candidate_kw(code: int) -> dict:
    """Transform parameters that realise a candidate code."""
    if code >= THIN_ONLY:
        return dict(select_mode=B.SELECT_HEURISTIC, thin_rows=THIN_ROWS,
                    max_depth=code - THIN_ONLY, flop_budget=THIN_BUDGET)
    if code == 0:
        return dict(select_mode=B.SELECT_NONE)
    return dict(select_mode=B.SELECT_FIXED, depth=code)


def collect(specs, reps: int = 3, with_heuristic: bool = True, log=None):
    """Features and measured log2 times (us) for every spec and candidate."""
    import matgen as mg
    X, y, group, hs = [], [], [], []
    for k, sp in enumerate(specs):
        A = mg.make_from_spec(sp)
        P = B.Plan(A.n, A.row_ptr, A.col, A.val)
        feats = B.sptrsv_costmodel_features(P.handle, CANDIDATES)
        for code, f in zip(CANDIDATES, feats):
            us = label_time(P, A.n, reps, **candidate_kw(code))
            X.append(f)
            y.append(np.log2(us))
            group.append(k)
        hs.append(np.log2(heuristic_time(P, A.n, reps)) if with_heuristic else np.nan)
        P.close()
        if log and (k % 20 == 0 or k == len(specs) - 1):
            log(f"collected {k + 1}/{len(specs)} (n={A.n})")
    return (np.asarray(X, np.float32), np.asarray(y, np.float32), np.asarray(group, np.int32),
            np.asarray(hs, np.float32))


def regret(model: CostModel, X, y, group, h_times):
    """Per matrix: time of the network's pick, of the best depth and of H."""
    rows = []
    pred = model.predict(X)
    for g in np.unique(group):
        sel = group == g
        yt, yp = y[sel], pred[sel]
        rows.append((2.0 ** yt[np.argmin(yp)], 2.0 ** yt.min(), 2.0 ** h_times[g],
                     2.0 ** yt[0]))
    r = np.asarray(rows)
    return dict(
        mean_regret=float(np.mean(r[:, 0] / r[:, 1])),
        geo_speedup_vs_heuristic=float(np.exp(np.mean(np.log(r[:, 2] / r[:, 0])))),
        geo_speedup_vs_plain=float(np.exp(np.mean(np.log(r[:, 3] / r[:, 0])))),
        geo_speedup_best_vs_heuristic=float(np.exp(np.mean(np.log(r[:, 2] / r[:, 1])))),
        picks_best=float(np.mean(r[:, 0] <= r[:, 1] * 1.0001)),
        matrices=int(r.shape[0]))


# --- per-segment network (SELECT_SEGMODEL) --------------------------------------

SEG_WEIGHTS_BIN = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "segmodel_weights.bin")
SEG_HIDDEN = 32
SEG_DMAX = 4
# segmentations timed per matrix: their new levels are the training rows
SEG_SELECTIONS = (
    ("plain", dict(select_mode=B.SELECT_NONE)),
    ("d1", dict(select_mode=B.SELECT_FIXED, depth=1)),
    ("d2", dict(select_mode=B.SELECT_FIXED, depth=2)),
    ("cp16", dict(select_mode=B.SELECT_CRITPATH, hop_weight=16, max_depth=4)),
    ("thin8", dict(select_mode=B.SELECT_HEURISTIC, thin_rows=THIN_ROWS, max_depth=8,
                   flop_budget=THIN_BUDGET)),
)
# the launch every segmentation is timed with (the staged kernel)
SEG_LAUNCH = dict(solve_mode=B.SOLVE_SYNCFREE, lanes_per_row=2, block_threads=128,
                  grid_blocks=0, tail_rows=-1, cta_run_rows=-1)


def seg_collect(specs, reps: int = 3, log=None):
    """Rows: the features of each new level of each timed segmentation and
    the log2 of the microseconds that level added (sptrsv_level_times);
    plus each plan's total time (us) per matrix and selection."""
    import torch
    import matgen as mg
    dev = torch.device("cuda", torch.cuda.current_device())
    X, y, group, totals = [], [], [], []
    for k, sp in enumerate(specs):
        A = mg.make_from_spec(sp)
        P = B.Plan(A.n, A.row_ptr, A.col, A.val)
        feat, ok = P.segment_features(SEG_DMAX)
        b = torch.ones(A.n, dtype=torch.float64, device=dev)
        tot = {}
        for name, kw in SEG_SELECTIONS:
            P.transform(**kw, **SEG_LAUNCH)
            first, depth = P.segments()
            us = P.level_times(b, reps)
            tot[name] = float(us.sum())
            for g, (t, d) in enumerate(zip(first, depth)):
                if d <= SEG_DMAX and ok[t, d]:
                    X.append(feat[t, d])
                    y.append(np.log2(max(float(us[g]), 0.02)))
                    group.append(k)
        totals.append(tot)
        P.close()
        if log:
            log(f"{k + 1}/{len(specs)} {sp['family']} n={A.n}: " +
                " ".join(f"{n} {v / 1e3:.3f}" for n, v in tot.items()))
    return (np.asarray(X, np.float32), np.asarray(y, np.float32), np.asarray(group, np.int32),
            totals)


def seg_evaluate(model: "CostModel", specs, reps: int = 7, log=None) -> dict:
    """On each matrix: the solve time of the network's segmentation
    (SELECT_SEGMODEL) against every timed segmentation (the exhaustive
    search over them: plain, depths 1 and 2, the critical-path selection, H
    on thin levels), one launch."""
    import matgen as mg
    B.sptrsv_segmodel_set_default(model.handle)
    rows = []
    try:
        for sp in specs:
            A = mg.make_from_spec(sp)
            P = B.Plan(A.n, A.row_ptr, A.col, A.val)
            t = {}
            for name, kw in SEG_SELECTIONS:
                P.transform(**kw, **SEG_LAUNCH)
                t[name] = time_solves(P, A.n, reps)
            P.transform(select_mode=B.SELECT_SEGMODEL, max_depth=SEG_DMAX, **SEG_LAUNCH)
            t["segmodel"] = time_solves(P, A.n, reps)
            P.close()
            best = min(v for k, v in t.items() if k != "segmodel")
            rows.append((t["segmodel"] / best, t["thin8"] / t["segmodel"],
                         t["plain"] / t["segmodel"], t["cp16"] / t["segmodel"]))
            if log:
                log(f"{sp['family']} n={A.n}: segmodel {t['segmodel']:.1f} us, best "
                    f"{best:.1f} us, regret {rows[-1][0]:.3f}")
    finally:
        B.sptrsv_segmodel_set_default(0)
    r = np.asarray(rows)
    geo = lambda a: float(np.exp(np.mean(np.log(a))))
    return dict(matrices=len(rows), geo_regret=geo(r[:, 0]), mean_regret=float(r[:, 0].mean()),
                within_5pct=float(np.mean(r[:, 0] <= 1.05)),
                geo_speedup_vs_thin_levels_h=geo(r[:, 1]), geo_speedup_vs_plain=geo(r[:, 2]),
                geo_speedup_vs_critpath=geo(r[:, 3]))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="costmodel")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--count", type=int, default=600)
    c.add_argument("--seed", type=int, default=5000)
    c.add_argument("--n-hi", type=float, default=5e5)
    c.add_argument("--reps", type=int, default=3)
    c.add_argument("--large", type=int, default=0,
                   help="collect this many larger matrices (training-only set) instead")
    c.add_argument("--out", required=True)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--train-frac", type=float, default=0.8)
    t.add_argument("--epochs", type=int, default=4000)
    t.add_argument("--lr", type=float, default=3e-3)
    t.add_argument("--extra", default=None,
                   help="additional training-only data (e.g. the larger matrices)")
    g = sub.add_parser("segmodel", help="collect, train and evaluate the per-segment network")
    g.add_argument("--count", type=int, default=40)
    g.add_argument("--seed", type=int, default=8000)
    g.add_argument("--train-frac", type=float, default=0.75)
    g.add_argument("--epochs", type=int, default=3000)
    g.add_argument("--lr", type=float, default=3e-3)
    g.add_argument("--data-out", default=None)
    g.add_argument("--out", default=SEG_WEIGHTS_BIN)
    g.add_argument("--large", action="store_true",
                   help="add eight large training-only matrices (segmodel_large_specs)")
    x = sub.add_parser("export", help="write weights as the library's network file")
    x.add_argument("--weights", default=WEIGHTS)
    x.add_argument("--out", default=WEIGHTS_BIN)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if args.cmd == "export":
        m = CostModel.load(args.weights)
        m.save(args.out)
        q = CostModel.load(args.out)
        assert np.array_equal(q.params(), m.params())
        print(args.out)
        return 0
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import matgen as mg
    if args.cmd == "segmodel":
        specs = mg.segmodel_specs(args.count, seed=args.seed)
        cut = int(round(len(specs) * args.train_frac))
        t0 = time.time()
        train = specs[:cut] + (mg.segmodel_large_specs() if args.large else [])
        X, y, g, totals = seg_collect(train, log=lambda s: print(s, flush=True))
        print(f"collected {len(y)} level rows from {len(train)} matrices in "
              f"{time.time() - t0:.1f} s")
        if args.data_out:
            np.savez(args.data_out, X=X, y=y, group=g,
                     totals=np.array([str(t) for t in totals]),
                     specs=np.array([str(s) for s in specs]))
        m = CostModel(n_in=B.SEG_FEATURES, hidden=SEG_HIDDEN)
        hist = m.fit(X, y, epochs=args.epochs, lr=args.lr, log_every=500)
        for e, l in hist:
            print(f"epoch {e}: train mse {l:.4f}")
        res = seg_evaluate(m, specs[cut:], log=lambda s: print(s, flush=True))
        big = seg_evaluate(m, [dict(index=0, family="stencil3d", n=128 ** 3, side=128, nrhs=1,
                                    seed=2000)], reps=5, log=lambda s: print(s, flush=True))
        res["stencil3d_128_regret"] = big["geo_regret"]
        res["train_mse_log2"] = float(hist[-1][1])
        print(json.dumps(res))
        m.save(args.out)
        return 0
    if args.cmd == "collect":
        if args.large:
            specs = mg.costmodel_large_specs(args.large)
        else:
            specs = mg.batch_specs(args.count, seed=args.seed, n_lo=1e4, n_hi=args.n_hi,
                                   nrhs_max=1, band_range=(5, 20))
        t0 = time.time()
        X, y, g, h = collect(specs, reps=args.reps, log=lambda s: print(s, flush=True))
        np.savez(args.out, X=X, y=y, group=g, h=h, candidates=np.array(CANDIDATES),
                 specs=np.array([str(s) for s in specs]))
        print(f"collected {len(specs)} matrices in {time.time() - t0:.1f} s")
        return 0
    d = np.load(args.data)
    X, y, g, h = d["X"], d["y"], d["group"], d["h"]
    ng = int(g.max()) + 1
    cut = int(round(ng * args.train_frac))
    tr, te = g < cut, g >= cut
    Xt, yt = X[tr], y[tr]
    if args.extra:
        e = np.load(args.extra)
        Xt, yt = np.concatenate([Xt, e["X"]]), np.concatenate([yt, e["y"]])
        print(f"training set: {int(tr.sum())} + {len(e['y'])} extra rows")
    m = CostModel()
    hist = m.fit(Xt, yt, epochs=args.epochs, lr=args.lr, log_every=500)
    for e, l in hist:
        print(f"epoch {e}: train mse {l:.4f}")
    te_mse = float(np.mean((m.predict(X[te]) - y[te]) ** 2))
    gt = g[te] - cut
    res = regret(m, X[te], y[te], gt, h[cut:])
    res["test_mse_log2"] = te_mse
    print(res)
    m.save(args.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())

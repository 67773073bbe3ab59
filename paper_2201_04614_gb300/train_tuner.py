"""Train the learned tuner on the GPU and evaluate it on held-out fields.

    python -m paper_2201_04614_gb300.train_tuner [--train 4000 --test 500]
        [--epochs 300] [--out paper_2201_04614_gb300/tuner_weights.bin]
        [--report tuner_eval.json]

Training fields are seeded synthetic fields (synth.tuner_field): rank 1-3,
2D/3D sides log-uniform in [64, 256], 1D lengths log-uniform in [64, 2^24],
spectral slopes in [-4, -1], noise up to 1e-2 of the range, ranges
log-uniform in [1e-3, 1e3], relative error bounds log-uniform in
[1e-5, 1e-2]; R = 512.  Each field is labelled by the exhaustive GPU sweep
(vsz_tuner_sweep: the cheapest class by estimated compressed size), its
features come from vsz_tuner_features, and the network is trained with the
library's gradient and Adam kernels.  Held-out fields (seeds after the
training seeds) measure what the tuned class saves over the default class
(block 256 / 16 / 8, zero padding), before and after the guard.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RADIUS = 512


def _gen_init():
    import synth.fields as sf
    sf._FFT_KW = {"workers": 1} if sf._FFT_KW else {}


def _gen(seed: int):
    import synth
    x, eb = synth.tuner_field(seed)
    return seed, np.ascontiguousarray(x.reshape(-1)), x.shape, eb


def fields(seeds, workers: int):
    """Yield (seed, flat x, dims, rel eb) in seed order, generated by a pool
    of spawned processes (started before any CUDA work in this process)."""
    if workers <= 1:
        for s in seeds:
            yield _gen(s)
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_gen_init) as pool:
        for r in pool.imap(_gen, seeds, chunksize=4):
            yield r


def label_fields(seeds, workers: int, log_every: int = 200):
    """Features, masks, sweep costs and outlier counts of each field."""
    import torch
    import paper_2201_04614_gb300 as vsz
    from paper_2201_04614_gb300 import tuner as T
    F, M, C, NO, dims_all = [], [], [], [], []
    t0 = time.time()
    for k, (seed, x, dims, eb) in enumerate(fields(seeds, workers)):
        p = vsz.Params.make(dims, 8, eb, "rel", RADIUS, "zero")
        xd = torch.from_numpy(x).cuda()
        _, f32 = T.features(p, xd)
        cost, nout = T.sweep(p, xd, with_nout=True)
        F.append(f32.cpu().numpy())
        C.append(cost.cpu().numpy())
        NO.append(nout.cpu().numpy())
        M.append(T.class_mask(len(dims)))
        dims_all.append(tuple(int(d) for d in dims))
        if log_every and (k + 1) % log_every == 0:
            print(f"[tuner] labelled {k + 1}/{len(seeds)} fields in {time.time() - t0:.0f}s", flush=True)
    return (np.array(F, np.float32), np.array(M, np.uint32), np.array(C, np.float64), np.array(NO, np.int64),
            dims_all)


def evaluate(net, X, masks, costs, nouts, dims, guard_fields=None):
    """Held-out metrics: accuracy against the sweep label and the estimated
    compressed size of the predicted / guarded / best class relative to the
    default class."""
    from paper_2201_04614_gb300 import tuner as T
    _, cls = net.forward(X, masks)
    pred = cls.cpu().numpy()
    n = len(pred)
    lab = np.array([T.label_of(c) for c in costs])
    dflt = np.array([T.default_class(len(d)) for d in dims])
    ar = np.arange(n)
    c_def, c_pred, c_best = costs[ar, dflt], costs[ar, pred], costs[ar, lab]
    rep = {
        "fields": n,
        "accuracy": float((pred == lab).mean()),
        "size_ratio_pred_vs_default_mean": float(np.mean(c_pred / c_def)),
        "size_ratio_best_vs_default_mean": float(np.mean(c_best / c_def)),
        "size_total_pred_vs_default": float(c_pred.sum() / c_def.sum()),
        "size_total_best_vs_default": float(c_best.sum() / c_def.sum()),
        "fields_pred_worse_than_default": int((c_pred > c_def).sum()),
        "nout_pred_le_default_frac": float(np.mean(nouts[ar, pred] <= nouts[ar, dflt])),
    }
    if guard_fields is not None:
        final = np.array([g["class"] for g in guard_fields])
        c_fin = costs[ar, final]
        rep.update({
            "size_ratio_guarded_vs_default_mean": float(np.mean(c_fin / c_def)),
            "size_total_guarded_vs_default": float(c_fin.sum() / c_def.sum()),
            "fields_guard_fell_back": int((final != pred).sum()),
            "nout_guarded_le_default_frac": float(np.mean(nouts[ar, final] <= nouts[ar, dflt])),
        })
    return rep, pred


def main(argv=None):
    """Generate the tuner's fields, label them by the GPU sweep, train, evaluate, save."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--test", type=int, default=500)
    ap.add_argument("--seed-base", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=max(1, min(14, (os.cpu_count() or 2) - 2)))
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)

    train_seeds = list(range(a.seed_base, a.seed_base + a.train))
    test_seeds = list(range(a.seed_base + a.train, a.seed_base + a.train + a.test))
    t0 = time.time()
    Xtr, Mtr, Ctr, Ntr, Dtr = label_fields(train_seeds, a.workers)
    Xte, Mte, Cte, Nte, Dte = label_fields(test_seeds, a.workers)
    t_label = time.time() - t0

    import torch
    import paper_2201_04614_gb300 as vsz
    from paper_2201_04614_gb300 import tuner as T
    ytr = np.array([T.label_of(c) for c in Ctr], np.int32)
    mu = Xtr.mean(axis=0)
    sigma = np.maximum(Xtr.std(axis=0), 1e-3)
    net = T.MLP(mu=mu, sigma=sigma, seed=1)
    t1 = time.time()
    hist = net.train(Xtr, ytr, Mtr, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=2, log_every=50)
    torch.cuda.synchronize()
    t_train = time.time() - t1

    # guard on the held-out fields (regenerated: the guard needs the data)
    guarded = []
    for (seed, x, dims, eb), f in zip(fields(test_seeds, a.workers), range(len(test_seeds))):
        p = vsz.Params.make(dims, 8, eb, "rel", RADIUS, "zero")
        xd = torch.from_numpy(x).cuda()
        guarded += T.choose([(p, xd)], mlp=net)
    rep_te, _ = evaluate(net, Xte, Mte, Cte, Nte, Dte, guarded)
    rep_tr, _ = evaluate(net, Xtr, Mtr, Ctr, Ntr, Dtr)
    label_hist = np.bincount(ytr, minlength=T.NCLASS).tolist()
    report = {
        "train_fields": a.train, "test_fields": a.test, "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
        "radius": RADIUS, "label_seconds": t_label, "train_seconds": t_train,
        "loss_first_epoch": float(hist[0]), "loss_last_epoch": float(hist[-1]),
        "train_label_histogram": label_hist, "train": rep_tr, "held_out": rep_te,
    }
    out = a.out or T.WEIGHTS_PATH
    net.save(out)
    print(json.dumps(report, indent=1), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()

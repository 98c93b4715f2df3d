"""Trains the per-round scheduler MLP on one GPU and evaluates it.

    python -m paper_2107_12720_gb300.train_scheduler [--out DIR] [--quick]

1. Training graphs: the R-MAT, planted and deep-cascade families of the
   benchmark workloads at other seeds and smaller sizes, each with G^T (all
   three variants) and without it (AC-6 / AC-3 only).
2. Labels: the exhaustive greedy per-round schedule (scheduler.greedy_judge).
3. Training: full-batch Adam with the library's CUDA kernels.
4. Evaluation on held-out graphs (the benchmark workloads themselves and the
   large mixed family, never used for training): device time of every fixed
   variant, the heuristic, the learned schedule and the judge's schedule.
Writes scheduler_mlp.npy (the model blob), judge_rows.npz (training data) and
scheduler_eval.json (the evaluation) to DIR (default: the package's models/).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import graphgen.configs as cfg  # noqa: E402
import paper_2107_12720_gb300 as P  # noqa: E402
from paper_2107_12720_gb300 import scheduler as S  # noqa: E402


def training_graphs(quick=False):
    """The benchmark families at other seeds and sizes (never the evaluation
    graphs): R-MAT scale 15..22 with several sink shares and skews, planted
    graphs of 1e5 and 1e6 vertices, deep cascades of 2^15..2^21 vertices and
    45..720 rounds, small batches and small mixed graphs."""
    gs = [cfg.rmat22(seed=101, scale=16), cfg.rmat22(seed=102, scale=17),
          graphgen.rmat(103, 16, 16, 0.57, 0.19, 0.19, 0.3, name="rmat16-sinks30"),
          graphgen.rmat(104, 15, 8, 0.45, 0.25, 0.15, 0.2, name="rmat15-ef8"),
          cfg.planted_trim(seed=105),
          cfg.deep_cascade(seed=106, log2n=15, n_chains=256),
          cfg.deep_cascade(seed=107, log2n=17, n_chains=2048),
          cfg.deep_cascade(seed=108, log2n=15, n_chains=128, literal=True),
          cfg.batched(seed=109, G=256, median=500.0, nmin=16, nmax=50000),
          cfg.rmat22(seed=110, scale=20),
          graphgen.rmat(111, 21, 16, 0.57, 0.19, 0.19, 0.05, name="rmat21-sinks5"),
          cfg.planted_trim(seed=112, nC=300000, nR=300000, nT=400000, t_sinks=20000),
          cfg.deep_cascade(seed=113, log2n=20, n_chains=4096),
          cfg.deep_cascade(seed=114, log2n=21, n_chains=2048),
          cfg.batched(seed=115, G=1024, median=1000.0, nmin=16, nmax=200000),
          cfg.large_mixed(seed=116, scale=18, block_log2=18, chain_len=500),
          cfg.rmat22(seed=117, scale=22),
          graphgen.rmat(118, 22, 12, 0.55, 0.2, 0.2, 0.2, name="rmat22-ef12-sinks20")]
    return gs[:4] if quick else gs


def eval_graphs(quick=False):
    """(name, graph, with G^T): the benchmark workloads themselves, held out."""
    gs = [("rmat22", cfg.config(1), True), ("deep_cascade_2^24", cfg.config(2), True),
          ("large_mixed_small", cfg.large_mixed(seed=5, scale=20, block_log2=19, chain_len=2000),
           True),
          ("planted_trim_noGT", cfg.config(0), False), ("rmat22_noGT", cfg.config(1), False)]
    return gs[:1] if quick else gs


def device_times(t, variant, reps=5):
    t.run(variant)
    return statistics.median(t.run(variant)["device_ms"] for _ in range(reps))


def collect(graphs, reps=2):
    rows = []
    for g in graphs:
        t0 = time.time()
        with P.Trimmer(g.off, g.tgt, flags=P.TRIM_FLAG_ROUND_LOG) as t:
            _, r_nog = S.greedy_judge(t, variants=(1, 2), reps=reps)   # without G^T
            t.run("ac4")                                                # builds G^T
            _, r_all = S.greedy_judge(t, variants=(0, 1, 2), reps=reps)
        rows += r_nog + r_all
        print(f"judge {g.name}: {len(r_all)} rounds, {time.time() - t0:.1f}s", flush=True)
    return rows


def evaluate(blob, quick=False, judge=True):
    out = {}
    for name, g, with_gt in eval_graphs(quick):
        with P.Trimmer(g.off, g.tgt, flags=P.TRIM_FLAG_ROUND_LOG) as t:
            fixed = ["ac4", "ac6", "ac3"] if with_gt else ["ac6", "ac3"]
            if with_gt:
                t.run("ac4")  # builds G^T; without it the variants are AC-6 and AC-3
            if name.startswith("deep"):
                fixed = [v for v in fixed if v != "ac3"]  # ~0.7 s per run, never competitive
            res = {v: device_times(t, v) for v in fixed + ["heuristic"]}
            t.set_model(blob)
            res["learned"] = device_times(t, "learned")
            t.run("learned")
            res["learned_rounds"] = [int(r.variant) for r in t.round_log()]
            if judge and len(res["learned_rounds"]) <= 64:
                sched, _ = S.greedy_judge(t, variants=(0, 1, 2) if with_gt else (1, 2), reps=2)
                t.set_schedule(np.asarray(sched, np.uint8))
                res["judge"] = device_times(t, "scripted")
                res["judge_rounds"] = sched
            best = min(res[v] for v in fixed)
            res["best_fixed"] = best
            res["gain_learned_vs_best_fixed"] = best / res["learned"]
            res["gain_learned_vs_heuristic"] = res["heuristic"] / res["learned"]
            res["with_GT"] = with_gt
            res["m"] = g.m
        hist = np.bincount(res["learned_rounds"], minlength=3).tolist()
        res["learned_rounds"] = hist
        out[name] = res
        print(name, {k: (round(v, 4) if isinstance(v, float) else v) for k, v in res.items()},
              flush=True)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=S.MODEL_DIR)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    os.makedirs(args.out, exist_ok=True)
    rows = collect(training_graphs(args.quick))
    X, y, w = S.rows_to_xy(rows)
    np.savez(os.path.join(args.out, "judge_rows.npz"), X=X, y=y, w=w,
             times=np.array([[tt.get(v, np.nan) for v in (0, 1, 2)] for _, tt in rows]),
             feats=np.array([f for f, _ in rows], np.float32))
    mean, istd = S.normalisation(X)
    Xn = (X - mean) * istd
    theta, hist = S.train(Xn, y, steps=args.steps, log_every=500)
    acc = float((S.predict(theta, Xn).argmax(axis=1) == y).mean())
    blob = S.make_blob(theta, mean, istd, X)
    S.save_blob(blob, os.path.join(args.out, "scheduler_mlp.npy"))
    print(f"trained on {len(y)} rounds (labels {np.bincount(y, minlength=3).tolist()}), "
          f"loss {hist[0][1]:.3f} -> {hist[-1][1]:.3f}, train accuracy {acc:.3f}", flush=True)
    ev = evaluate(blob, args.quick)
    json.dump({"train_rows": int(len(y)), "label_counts": np.bincount(y, minlength=3).tolist(),
               "loss_history": hist, "train_accuracy": acc, "eval": ev},
              open(os.path.join(args.out, "scheduler_eval.json"), "w"), indent=1)


if __name__ == "__main__":
    main()

"""Per-round scheduler: labelled round logs, GPU training, model files.

The learned scheduler (TRIM_SCHED_LEARNED) is a 12 -> 32 -> 32 -> 3 ReLU MLP run
by one warp between rounds. This module produces its training data and trains
it with the library's own CUDA kernels (trim_mlp_loss_grad, trim_mlp_adam_step):

  greedy_judge   the exhaustive per-round schedule: at every round r it runs the
                 scripted schedule (best prefix so far) + [X kept to the end] for
                 X in AC-4, AC-6, AC-3, charges X the device time of the rounds it
                 would run (round log), and keeps the cheapest. Its per-round
                 choices are the labels; the features the kernel recorded for
                 round r are the inputs.
  train          full-batch Adam on the GPU, softmax cross-entropy.
  make_blob      weights + input normalisation + training range, the layout
                 trim_set_model expects (features outside the range fall back to
                 the heuristic in the kernel).

Feature vector of round r+1 (computed on the device after round r):
  0 log2(1+|F_r|)   1 log2(1+sum indeg F_r)
  2 log2(1+in-edges of removed vertices that AC-4 has not pushed yet)
  3 log2(1+n_live)  4 log2(1+m_live)          5 |F_r| / n_live
  6 sum indeg F_r / m_live                    7..9 fractions of F_r with in-degree
  <8, <256, >=256   10 log2(1 + ns per frontier vertex of round r-1)
  11 the variant of round r (whose state is warm; -1 before round 1).
m_live is the number of edges between live vertices when G^T is present (m
minus the in-edges of removed vertices) and the number of out-edges of live
vertices without it. The in-degree features are 0 without G^T.
"""
from __future__ import annotations

import os

import numpy as np

from . import abi
from .abi import TRIM_MLP_NIN, TRIM_MLP_NPARAMS

FEATURES = ["log2_frontier", "log2_in_edges", "log2_ac4_backlog", "log2_n_live", "log2_m_live",
            "frontier_over_live", "in_edges_over_m_live", "frac_indeg_lt8", "frac_indeg_lt256",
            "frac_indeg_ge256", "log2_ns_per_vertex_prev", "current_variant"]
MODEL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models")
MODEL_PATH = os.path.join(MODEL_DIR, "scheduler_mlp.npy")


def round_times(trimmer):
    """[(round, variant, device seconds, features)] of the last logged run."""
    return [(r.round, r.variant, (r.t_end_ns - r.t_start_ns) * 1e-9, list(r.features))
            for r in trimmer.round_log()]


def run_scripted(trimmer, schedule, reps=1):
    """Runs a scripted schedule `reps` times; per-round min device times and the
    features of the last run."""
    trimmer.set_schedule(np.asarray(schedule, np.uint8))
    best = None
    feats = None
    for _ in range(reps):
        trimmer.run("scripted")
        rt = round_times(trimmer)
        t = np.array([x[2] for x in rt])
        best = t if best is None else np.minimum(best, t)
        feats = [x[3] for x in rt]
    return best, feats


def greedy_judge(trimmer, variants=(0, 1, 2), reps=2, horizon=None):
    """The exhaustive per-round schedule of the graph behind `trimmer` (a Trimmer
    created with TRIM_FLAG_ROUND_LOG): at every round r, for each variant X it runs
    (best prefix so far) + [X] kept for the rest of the run, and charges X the
    device time of rounds r .. r+horizon-1 (default: to the end). A horizon of
    1 is the plain greedy rule, which never pays a one-time entry cost (AC-6's
    set build, AC-4's backlog); the rollout charges those costs against the
    rounds they serve. The prefix of chosen variants only ever improves on the
    best fixed variant (round 1's choice is the best variant kept to the end).
    Returns (schedule, rows) with rows[r-1] = (features used for round r,
    {X: charged time})."""
    trimmer.set_schedule(np.asarray([variants[0]], np.uint8))
    trimmer.run("scripted")  # warm-up, and alpha
    alpha = len(trimmer.round_log())
    prefix = []
    rows = []
    for r in range(1, alpha + 1):
        times = {}
        feats = None
        for x in variants:
            t, f = run_scripted(trimmer, prefix + [x] * (alpha - r + 1), reps)
            end = alpha if horizon is None else min(alpha, r - 1 + horizon)
            times[x] = float(np.sum(t[r - 1:end]))
            if x == variants[0] or feats is None:
                feats = f[r - 1]
        best = min(times, key=times.get)
        prefix.append(best)
        rows.append((feats, times))
    return prefix, rows


def rows_to_xy(rows, min_gap=0.05):
    """Features and argmin labels; rounds whose best two variants are within
    `min_gap` (relative) are dropped as ambiguous."""
    X, y, w = [], [], []
    for feats, times in rows:
        order = sorted(times, key=times.get)
        t0, t1 = times[order[0]], times[order[1]] if len(order) > 1 else float("inf")
        if t1 < float("inf") and (t1 - t0) < min_gap * t0:
            continue
        X.append(feats)
        y.append(order[0])
        w.append(t1 - t0)
    return np.asarray(X, np.float32).reshape(-1, TRIM_MLP_NIN), np.asarray(y, np.uint8), np.asarray(w)


def he_init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (the random numbers are drawn here, on the
    host, and passed to the device as the initial parameters)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / 12), (32, 12)), np.zeros(32),
             rng.normal(0, np.sqrt(2.0 / 32), (32, 32)), np.zeros(32),
             rng.normal(0, np.sqrt(2.0 / 32), (3, 32)), np.zeros(3)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def normalisation(X):
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    istd = np.where(std > 1e-6, 1.0 / np.maximum(std, 1e-6), 1.0)
    return mean.astype(np.float32), istd.astype(np.float32)


def train(X, y, steps=2000, lr=3e-3, seed=0, log_every=0):
    """Full-batch Adam on the GPU with the library's kernels. X must already be
    normalised. Returns (parameters, loss history)."""
    import torch
    N = X.shape[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    theta = dev(he_init(seed))
    dX, dy = dev(X.astype(np.float32)), dev(y.astype(np.uint8))
    grad = torch.empty(TRIM_MLP_NPARAMS, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(abi.trim_mlp_scratch_bytes(N) // 4 + 1, dtype=torch.float32,
                          device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hist = []
    for t in range(1, steps + 1):
        abi.trim_mlp_loss_grad(theta, dX, dy, N, loss, grad, scratch, stream)
        abi.trim_mlp_adam_step(theta, grad, m, v, t, lr, 0.9, 0.999, 1e-8, stream)
        if log_every and (t % log_every == 0 or t == 1):
            hist.append((t, float(loss.item())))
    abi.trim_mlp_loss_grad(theta, dX, dy, N, loss, grad, scratch, stream)
    hist.append((steps, float(loss.item())))
    return theta.cpu().numpy(), hist


def predict(theta, Xn):
    import torch
    N = Xn.shape[0]
    dt = torch.from_numpy(np.ascontiguousarray(theta, np.float32)).cuda()
    dX = torch.from_numpy(np.ascontiguousarray(Xn, np.float32)).cuda()
    out = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    abi.trim_mlp_forward(dt, dX, N, out, torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy()


# features that are log2 of a size (frontier, edges, live counts, time per
# vertex): the model may extrapolate them to larger or smaller graphs, by up to
# LOG2_MARGIN binary orders of magnitude outside the training range
LOG2_FEATURES = (0, 1, 2, 3, 4, 10)
LOG2_MARGIN = 8.0


def make_blob(theta, mean, istd, X, margin=0.25):
    """Model blob for trim_set_model: parameters, normalisation, and the range
    in which the kernel trusts the model (outside it the heuristic decides): the
    training range of every feature widened by `margin` of its span, and the
    size features (log2) by LOG2_MARGIN more."""
    lo, hi = X.min(axis=0), X.max(axis=0)
    span = np.maximum(hi - lo, 1e-3)
    lo, hi = lo - margin * span, hi + margin * span
    for i in LOG2_FEATURES:
        lo[i] -= LOG2_MARGIN
        hi[i] += LOG2_MARGIN
    return np.concatenate([theta, mean, istd, lo, hi]).astype(np.float32)


def save_blob(blob, path=MODEL_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, np.asarray(blob, np.float32))


def load_blob(path=MODEL_PATH):
    return np.load(path).astype(np.float32)

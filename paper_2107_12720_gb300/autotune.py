"""Autotuner for the launch shape and the scheduler thresholds (trim_params_t).

    python -m paper_2107_12720_gb300.autotune --config 1 [--small] [--variants ac4,learned]
                                               [--out DIR/tuned_params.json]

For one workload it times every point of a small search space with the
library's own device timer (median of `reps` complete runs after one warm-up)
and keeps, per variant, the fastest point:

  block_threads      128, 256, 384, 512 threads per persistent CTA
  ctas_per_sm        as many as fit (0), or 1
  heur_push_ratio    0.5, 1, 2    (heuristic / learned fallback: AC-4 vs the rest)
  heur_ac6_ratio     0.5, 1, 2    (heuristic without G^T: AC-6 vs AC-3)
  sched_commit_rounds 4, 8, 32    (scheduled runs: rounds before a commit)
  local_round_edges  0, 2^14, 2^18, 2^20 (AC-4: pending in-edges up to which rounds
                     run CTA-locally)

The launch shape is searched for every variant; the scheduler thresholds only
for the heuristic and learned schedules (for which the launch shape is taken
from AC-4's best point first). The result file maps "<workload>/<variant>" to
the chosen trim_params_t fields plus the measured times; `apply` sets them on a
Trimmer. Every run stays exact: the parameters change speed, never results.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from . import scheduler as S  # noqa: E402

TUNED_PATH = os.path.join(S.MODEL_DIR, "tuned_params.json")

LAUNCH_SPACE = {"block_threads": (128, 256, 384, 512), "ctas_per_sm": (0, 1)}
MIN_GAIN = 0.02  # a point must beat the best so far by 2% (timing noise is ~0.5%)
SCHED_SPACE = {"heur_push_ratio": (0.5, 1.0, 2.0), "heur_ac6_ratio": (0.5, 1.0, 2.0),
               "sched_commit_rounds": (4, 8, 32)}
LOCAL_SPACE = {"local_round_edges": (0, 1 << 14, 1 << 18, 1 << 20)}


def _points(space):
    keys = list(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        yield dict(zip(keys, vals))


def time_point(trimmer, variant, params, reps=5):
    """Median device time (ms) of `reps` runs of `variant` with `params` applied
    on top of the library defaults."""
    trimmer.set_params(**{**default_params(), **params})
    trimmer.run(variant)
    return statistics.median(trimmer.run(variant)["device_ms"] for _ in range(reps))


def default_params():
    from . import abi
    p = abi.trim_default_params()
    return {k: getattr(p, k) for k, _ in abi.TrimParams._fields_}


def tune(trimmer, variants=("ac4", "ac6", "ac3", "heuristic", "learned"), reps=5, log=None):
    """Returns {variant: {"params": best, "ms": best_ms, "default_ms": ms}}."""
    out = {}
    base = time_point(trimmer, "ac4", {}, reps) if "ac4" in variants else None
    best_launch = {}
    for v in variants:
        default_ms = base if (v == "ac4" and base is not None) else time_point(trimmer, v, {}, reps)
        best, best_ms = {}, default_ms
        for p in _points(LAUNCH_SPACE):
            ms = time_point(trimmer, v, p, reps)
            if log:
                log(f"{v:9s} {p} {ms:.4f} ms")
            if ms < best_ms * (1.0 - MIN_GAIN):
                best, best_ms = p, ms
        if v in ("ac4", "heuristic", "learned"):  # AC-4 runs (and committed AC-4 stretches)
            for p in _points(LOCAL_SPACE):
                q = {**best, **p}
                ms = time_point(trimmer, v, q, reps)
                if log:
                    log(f"{v:9s} {q} {ms:.4f} ms")
                if ms < best_ms * (1.0 - MIN_GAIN):
                    best, best_ms = q, ms
        if v == "ac4":
            best_launch = dict(best)
        if v in ("heuristic", "learned"):
            launch = dict(best_launch or best)
            for p in _points(SCHED_SPACE):
                q = {**launch, **p}
                ms = time_point(trimmer, v, q, reps)
                if log:
                    log(f"{v:9s} {q} {ms:.4f} ms")
                if ms < best_ms * (1.0 - MIN_GAIN):
                    best, best_ms = q, ms
        out[v] = {"params": best, "ms": best_ms, "default_ms": default_ms}
    trimmer.set_params(**default_params())
    return out


class _Batched:
    """A context whose runs are batched runs over fixed graph offsets."""

    def __init__(self, t, graph_off):
        self.t, self.graph_off = t, graph_off

    def set_params(self, **kw):
        self.t.set_params(**kw)

    def run(self, variant):
        return self.t.batch_run(self.graph_off, variant)


def load(path=TUNED_PATH):
    return json.load(open(path)) if os.path.exists(path) else {}


def save(entries, path=TUNED_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    old = load(path)
    old.update(entries)
    json.dump(old, open(path, "w"), indent=1, sort_keys=True)


def apply(trimmer, workload: str, variant: str, path=TUNED_PATH) -> dict:
    """Sets the tuned parameters of (workload, variant) on `trimmer`, if any;
    returns them ({} when none were tuned)."""
    entry = load(path).get(f"{workload}/{variant}")
    params = entry["params"] if entry else {}
    if params:
        trimmer.set_params(**{**default_params(), **params})
    return params


def main(argv=None):
    import numpy as np
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--variants", default="ac4,ac6,ac3,heuristic,learned")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=TUNED_PATH)
    args = ap.parse_args(argv)
    import torch
    import graphgen.configs as cfg
    import paper_2107_12720_gb300 as P
    torch.cuda.set_device(0)
    g = cfg.config_small(args.config) if args.small else cfg.config(args.config)
    key = f"config{args.config}{'-small' if args.small else ''}"
    variants = [v for v in args.variants.split(",") if v]
    with P.Trimmer(g.off, g.tgt) as t:
        if os.path.exists(S.MODEL_PATH):
            t.set_model(np.load(S.MODEL_PATH))
        target = t
        if args.config == 3 and g.graph_off is not None:  # the batched workload: batched runs
            target = _Batched(t, np.asarray(g.graph_off, np.uint32))
        res = tune(target, variants, args.reps, log=lambda s: print(s, flush=True))
    save({f"{key}/{v}": r for v, r in res.items()}, args.out)
    for v, r in res.items():
        print(f"{key}/{v}: {r['ms']:.4f} ms (defaults {r['default_ms']:.4f} ms) with {r['params']}",
              flush=True)


if __name__ == "__main__":
    main()

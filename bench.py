"""Benchmark: trimming throughput (edges/s = m / trim time) on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config I] [--variant V] [--no-sweep] [--no-extra]

A step is one complete trimming (every round, from the initial sink pass to the
empty frontier) of the large mixed workload (configs index 4: R-MAT scale 26
union a 2^25-vertex planted block with ~10,000-deep chains; n = 100.7M,
m = 1.22e9, alpha = 10,004) with inputs resident in HBM, run with the learned
per-round scheduler; the fixed variants and the heuristic are timed beside it
on the same graph, and the R-MAT scale-22 workload (index 1) and the batched
workload (index 3, one replayed CUDA graph against each graph trimmed alone)
ride along as extra keys. The L2 cache is flushed before every step and the
step is timed with CUDA events on the library's stream. Rank 0 prints one
JSON line.

--impl reference times the CPU oracle (sequential queue peeling, Algorithm 5
run one step at a time) on the host on the same full workload graph.
N > 1: independent replicas, one per GPU (trimming one graph has no sharded
form here; see the design notes), value = edges of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s (m/trim time) at 1 GB300, % HBM roofline; learned/batched vs fixed schedule"
UNIT = "edges/s"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "trim_persistent_kernel_rmat22.txt")
REFERENCE_BUDGET_S = 150.0  # wall-clock bound of the reference arm's timed steps
KERNEL_SRC = os.path.join(ROOT, "paper_2107_12720_gb300", "csrc", "trim_kernels.cu")


# ---------------------------------------------------------------- workload

def workload(idx: int, small: bool = False):
    import graphgen.configs as cfg
    if small:  # the same recipe at the sizes of the parity tests (profiling captures)
        g = cfg.config_small(idx)
        return g, f"small case of config {idx}: {g.name} (n={g.n}, m={g.m})"
    g = cfg.config(idx)
    names = {0: "planted_trim n=100,000 (C 30k / R 30k / T 40k), seed 1",
             1: "rmat22: R-MAT scale 22 (n=4,194,304), edge factor 16, a/b/c=.57/.19/.19, "
                "ids permuted, dedup, no self-loops, 10% sinks, seed 2",
             2: "deep_cascade n=2^24: C 10% / R 20% / T 70% as 4,096 chains (~2,867 deep), "
                "mean out-degree 8, seed 3",
             3: "batched: 4,096 planted graphs, log-normal sizes (median 2,000, sigma 1.5), seed 4",
             4: "large_mixed: R-MAT scale 26 + 2^25 planted block (chains ~10,000 deep), seed 5"}
    return g, names[idx]


def host_transpose(off: np.ndarray, tgt: np.ndarray):
    """G^T as plain data preparation (the workloads supply both CSRs)."""
    import graphgen
    return graphgen.transpose(off, tgt)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, period_ms: int = 100):
        self.dev = device_index
        self.period = period_ms
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.6)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        # samples under load: the upper half of the observed clocks (the run keeps the GPU busy)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline

def algorithmic_bytes(n: int, st: dict, variant_flags: dict) -> int:
    """Bytes the method must move in one run (per-unit figures of the design
    notes): init 12n; per removed vertex 20 B (log write + read, level write,
    G^T offsets); AC-4 12 B per in-edge (id read + 8-byte atomic read-modify-
    write); AC-3 12 B per live-list entry swept plus 4 B per survivor written;
    AC-6 24 B per supporting-set member re-scanned; 8 B per out-edge inspected
    (target id + its level)."""
    D = st["n_dead"]
    b = 12 * n + 20 * D
    b += 12 * st["in_edges_pushed"]
    b += 16 * st["live_swept"]
    b += 24 * st["candidates"]
    b += 8 * st["edges_inspected"]
    return int(b)


def atomic_ceiling(P, t, off_in, tgt_in, pushed: int, cap: int = 32 << 20):
    """L2 atomic ceiling of the AC-4 pushes of the last run: the counter indices
    the run decremented (the in-edges of its removed vertices, at most `cap` of
    them, in removal-agnostic vertex order) replayed by one fully parallel kernel
    of returning atomicSub (trim_probe_atomic_rate). Returns (ops/s, indices)."""
    import torch
    if pushed <= 0:
        return None, 0
    lvl = t.level(device=False)
    dead = np.nonzero(lvl != P.TRIM_LIVE)[0]
    starts = off_in[dead].astype(np.int64)
    lens = off_in[dead + 1].astype(np.int64) - starts
    keep = np.searchsorted(np.cumsum(lens), cap, side="right")
    starts, lens = starts[:keep], lens[:keep]
    total = int(lens.sum())
    if total == 0:
        return None, 0
    shift = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    idx = tgt_in[np.arange(total, dtype=np.int64) + shift].astype(np.uint32)
    d_idx = torch.from_numpy(idx.view(np.int32)).cuda()
    d_cnt = torch.empty(len(lvl), dtype=torch.int32, device="cuda")
    ms = P.abi.trim_probe_atomic_rate(d_idx.data_ptr(), total, d_cnt.data_ptr(), len(lvl), 5,
                                      torch.cuda.current_stream().cuda_stream)
    return total / (ms * 1e-3), total


def measured_peaks(path: str = None):
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json at the repository
    root, else the 6.8 TB/s fallback; an unreadable file or a missing or
    non-positive `hbm_gbs` also gives the fallback (the benchmark still runs)."""
    p = path or os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback"


def kernel_source_sha() -> str:
    """Hash of the kernel source's code: comment-only lines and blank lines are
    left out, so that editing a comment does not orphan a profile."""
    lines = [ln.rstrip() for ln in open(KERNEL_SRC, encoding="utf-8")]
    code = "\n".join(ln for ln in lines if ln.strip() and not ln.strip().startswith("//"))
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def _profile_fields(path: str) -> dict:
    kv = {}
    for line in open(path, encoding="utf-8"):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip().split()[0] if v.strip() else ""
    return kv


def profiled_traffic(config: int, small: bool, schedule: str):
    """DRAM bytes per run of the persistent kernel(s) from a committed ncu
    summary under profiles/ that covers this workload (workload_config, small)
    and schedule and was taken on the current kernel source; else None. The
    summary of the R-MAT scale-22 AC-4 run predates the workload keys and
    covers (1, full size, ac4)."""
    sha = kernel_source_sha()
    pdir = os.path.dirname(PROFILE_TRAFFIC)
    if not os.path.isdir(pdir):
        return None
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".txt"):
            continue
        path = os.path.join(pdir, name)
        kv = _profile_fields(path)
        if path == PROFILE_TRAFFIC and "workload_config" not in kv:
            kv.update(workload_config="1", small="0", schedule="ac4")
        if kv.get("workload_config") != str(config) or kv.get("small", "0") != str(int(small)) \
                or kv.get("schedule") != schedule or kv.get("kernel_source_sha") != sha:
            continue
        for key in ("dram_bytes_per_run", "dram_bytes_per_launch"):
            try:
                return int(float(kv[key]))
            except (KeyError, ValueError):
                pass
    return None


# ---------------------------------------------------------------- distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """Maximum of a per-rank scalar over all ranks (the slowest rank's time)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- CPU baseline

def cpu_baseline(g, csr_in, seconds: float = 12.0) -> dict:
    """The oracle (sequential C, one thread) on the same graph, G^T given as
    input (prepared outside the timing, as for the GPU), repeated for about
    `seconds` (at least 3 runs)."""
    import oracle
    times = []
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end or len(times) < 3:
        t0 = time.perf_counter()
        oracle.peel(g.off, g.tgt, csr_in)
        times.append(time.perf_counter() - t0)
    mean = statistics.mean(times)
    return {"value": g.m / mean, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the full workload graph, {len(times)} runs of the single-threaded "
                      f"oracle peel (G^T given as input), mean {mean * 1e3:.1f} ms",
            "cpu": cpu_name(), "nproc": os.cpu_count()}


def cpu_name() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def reference_steps(t_one: float, steps: int, warmup: int, budget: float):
    """(warm-up runs, timed runs) of the reference arm: the requested ones when
    they fit the wall-clock budget, else as many as fit (the first, untimed
    run counts as one warm-up; at least one timed run)."""
    if t_one * (steps + max(0, warmup - 1)) <= budget:
        return max(0, warmup - 1), steps
    fit = max(1, int(budget / max(t_one, 1e-9)))
    return 0, min(steps, fit)


def run_reference(args, rank, ws):
    if rank != 0:
        return
    import oracle
    g, wname = workload(args.config, args.small)
    csr_in = host_transpose(g.off, g.tgt)
    # every step is one oracle run over the full workload graph; when the
    # requested steps would take longer than REFERENCE_BUDGET_S, fewer steps are
    # timed (stated in the sample), never a different graph
    t0 = time.perf_counter()
    oracle.peel(g.off, g.tgt, csr_in)
    t_one = time.perf_counter() - t0
    n_warm, n_steps = reference_steps(t_one, args.steps, args.warmup, REFERENCE_BUDGET_S)
    for _ in range(n_warm):
        oracle.peel(g.off, g.tgt, csr_in)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        oracle.peel(g.off, g.tgt, csr_in)
    dt = time.perf_counter() - t0
    value = g.m * n_steps / dt
    sample = f"the full workload graph per step, {n_steps} timed steps after {n_warm + 1} untimed"
    if n_steps < args.steps:
        sample += (f" ({args.steps} requested: one run takes {t_one:.1f} s, the timed steps are "
                   f"capped at {REFERENCE_BUDGET_S:.0f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": n_steps, "warmup": n_warm + 1, "requested_steps": args.steps,
            "ms_per_step": dt / n_steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": wname, "n": g.n, "m": g.m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu": cpu_name(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def tuned_key(config: int, small: bool) -> str:
    return f"config{config}{'-small' if small else ''}"


def apply_tuned(t, args, variant, key=None):
    """Autotuned trim_params_t of this workload and variant (the autotuner's
    result file), unless --no-tuned or none were tuned; returns them."""
    if args.no_tuned:
        return {}
    from paper_2107_12720_gb300 import autotune
    return autotune.apply(t, key or tuned_key(args.config, args.small), variant)


def restore_defaults(t):
    from paper_2107_12720_gb300 import autotune
    t.set_params(**autotune.default_params())


def time_variant(P, t, variant, steps, warmup, flush_buf, graph_off=None):
    """Device time of `steps` complete trims (L2 flushed before each). With
    graph_off the step is one batched trim (trim_batch_run, a replayed CUDA
    graph) of all packed graphs."""
    import torch
    stream = t.stream
    run = (lambda: t.batch_run(graph_off, variant)) if graph_off is not None else None
    if variant == "inout":  # in+out trimming (another problem on the same graph)
        run = t.run_inout
    for _ in range(warmup):
        run() if run else t.run(variant)
    times, kern = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    last = None
    # every schedule is enqueued asynchronously: a fixed variant as one
    # persistent launch, a scheduled one as its first kernel plus the
    # all-variant continuation behind it; a batched run through trim_batch_run
    launches = 0
    for _ in range(steps):
        flush_buf.add_(1)  # writes more than the L2 holds, on the same stream
        e0.record(stream)
        if run:
            last = run()
            e1.record(stream)
        else:
            t.run_async(variant)
            e1.record(stream)
            last = t.sync()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kern.append(last["device_ms"])
        launches += last["launches"]  # reset, persistent kernel(s), continuation
    last = dict(last, launches=launches)
    return times, kern, last


def sweep_variants(P, t, g, args, key, names, flush, gofs=None, label=""):
    """Times every schedule in `names` on the context `t` (tuned parameters of
    `key` applied per schedule, library defaults restored afterwards)."""
    out = {}
    for v in names:
        tuned_v = apply_tuned(t, args, v, key)
        # a batched fixed variant is captured into a CUDA graph on its second
        # call: two warm-up calls keep the capture out of the timed steps
        ts, ks, st = time_variant(P, t, v, max(args.sweep_steps, args.steps // 10),
                                  2 if gofs is not None else 1, flush, gofs)
        restore_defaults(t)
        out[v] = {"ms": statistics.mean(ts), "kernel_ms": statistics.mean(ks),
                  "ms_ci95": (1.96 * statistics.stdev(ts) / len(ts) ** 0.5)
                  if len(ts) > 1 else None,
                  "params": tuned_v or "defaults",
                  "edges_per_s": g.m / (statistics.mean(ts) * 1e-3),
                  "rounds_by_variant": st["rounds_by_variant"], "segments": st["segments"],
                  "async_from_round": st.get("async_round", 0)}
        print(f"# {label}{v:10s} {statistics.mean(ts):8.4f} ms  kernel {statistics.mean(ks):8.4f} ms"
              f"  {g.m / statistics.mean(ts) / 1e-3:.3e} edges/s  rounds {st['rounds_by_variant']}"
              f"  segments {st['segments']}", file=sys.stderr, flush=True)
    return out


def schedules_summary(sweep: dict) -> dict:
    """Best fixed variant of a sweep and every schedule's speed relative to it
    (> 1: faster than the best fixed variant)."""
    fixed = {v: sweep[v]["ms"] for v in ("ac4", "ac6", "ac3") if v in sweep}
    if not fixed:
        return {}
    best = min(fixed, key=fixed.get)
    out = {"best_fixed": best, "best_fixed_ms": fixed[best]}
    for v in ("heuristic", "learned"):
        if v in sweep:
            out[f"{v}_vs_best_fixed"] = fixed[best] / sweep[v]["ms"]
    return out


def per_graph_fixed(P, g, variant="ac4", limit=None):
    """The unbatched schedule: every packed graph trimmed alone with one fixed
    variant (one context per graph, G^T given); returns the summed device time
    (context creation and copies excluded) and the graphs timed."""
    go = g.graph_off.astype(np.int64)
    total_ms, count = 0.0, 0
    idx = range(len(go) - 1) if limit is None else range(0, len(go) - 1, max(1, (len(go) - 1) // limit))
    for gi in idx:
        a, b = int(go[gi]), int(go[gi + 1])
        off = (g.off[a:b + 1] - g.off[a]).astype(np.uint32)
        tgt = (g.tgt[g.off[a]:g.off[b]] - a).astype(np.uint32)
        oi, ti = host_transpose(off, tgt)
        with P.Trimmer(off, tgt, oi, ti) as t:
            t.run(variant)
            total_ms += t.run(variant)["device_ms"]
        count += 1
    scale = (len(go) - 1) / count
    return total_ms * scale, count


def touched_input_bytes(n: int, st: dict) -> int:
    """Bytes of distinct CSR entries the kernels read from host memory in place
    (TRIM_MEM_HOST_MAPPED), from the run's work counters: the initial pass reads
    both offset arrays whole; AC-4 reads the G^T row of every pushed in-edge;
    AC-6/AC-3 read the target of every out-edge they inspect."""
    return 8 * (n + 1) + 4 * int(st["in_edges_pushed"]) + 4 * int(st["edges_inspected"])


def e2e_measure(P, g, off_in, tgt_in, variant, steps, graph_off=None, mapped=True, params=None,
                model=None):
    """Through the C ABI with host buffers, host wall clock around the whole
    call sequence: trim_create on page-locked host CSR (and G^T), trim_run,
    trim_level into a host array, trim_destroy. mapped: the kernels read the
    host CSR in place over the CPU-GPU link (TRIM_MEM_HOST_MAPPED); otherwise
    trim_create first copies it to device memory (TRIM_MEM_HOST)."""
    import torch
    pin = lambda a: torch.from_numpy(a.view(np.int32)).pin_memory()
    ho, ht, hoi, hti = pin(g.off), pin(g.tgt), pin(off_in), pin(tgt_in)
    out = torch.empty(g.n, dtype=torch.int32).pin_memory()
    ts = []
    for s in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with P.Trimmer(ho, ht, hoi, hti, host_mapped=mapped) as t:
            if params:
                t.set_params(**params)
            if model is not None:
                t.set_model(model)
            t.batch_run(graph_off, variant) if graph_off is not None else t.run(variant)
            P.trim_level(t.ctx, out.data_ptr(), 0)
        t1 = time.perf_counter()
        if s:  # the first call pays one-time costs (module load, context)
            ts.append(t1 - t0)
    copied = (g.off.nbytes + g.tgt.nbytes + off_in.nbytes + tgt_in.nbytes)
    del ho, ht, hoi, hti
    return g.m / statistics.mean(ts), copied, out.numel() * 4


def split_by_size(P, g, args, flush, stream, max_n=4096, max_m=65536, steps=20):
    """Bound on what trimming the small graphs of a batch apart (one CTA each,
    from a device-side queue) could save: the batched AC-4 time of the union
    of only the graphs above one CTA's capacity (max_n vertices or max_m
    edges), and of only the small ones, next to the whole union. Even if the
    small graphs cost nothing elsewhere, a split saves at most
    union - union_of_large_graphs."""
    import torch
    import graphgen
    go = g.graph_off.astype(np.int64)
    parts, small = [], []
    for gi in range(len(go) - 1):
        a, b = int(go[gi]), int(go[gi + 1])
        off = (g.off[a:b + 1] - g.off[a]).astype(np.uint32)
        tgt = (g.tgt[g.off[a]:g.off[b]] - a).astype(np.uint32)
        parts.append(graphgen.Graph(off, tgt))
        small.append((b - a) <= max_n and int(off[-1]) <= max_m)
    out = {"max_n": max_n, "max_m": max_m, "small_graphs": int(sum(small)),
           "small_edges_share": sum(p.m for p, s_ in zip(parts, small) if s_) / g.m}
    for name, sel in (("union_of_large_graphs", [not x for x in small]),
                      ("union_of_small_graphs", small)):
        u = graphgen.union([p for p, s_ in zip(parts, sel) if s_])
        oi, ti = host_transpose(u.off, u.tgt)
        dev = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
        with P.Trimmer(dev(u.off), dev(u.tgt), dev(oi), dev(ti), stream=stream) as t:
            apply_tuned(t, args, "ac4", tuned_key(3, False))
            ts, ks, st = time_variant(P, t, "ac4", steps, 2, flush, u.graph_off)
        out[name] = {"ms": statistics.mean(ts), "rounds": st["rounds"], "m": u.m}
        print(f"# [3] {name}: {statistics.mean(ts):.4f} ms rounds {st['rounds']} m {u.m}",
              file=sys.stderr, flush=True)
    return out


def scc_timing(t, g, steps=3):
    """SCC decomposition of the graph (trim_run_scc: in+out trimming, size-2
    trimming, forward-backward steps), elapsed time on the stream."""
    t.run_scc(device=True)
    runs = [t.run_scc(device=True)[1] for _ in range(steps)]
    last = runs[-1]
    out = dict(last, ms=statistics.mean(r["ms"] for r in runs))
    print(f"# scc: {out['ms']:.3f} ms, {last['components']} components, steps {last['fwbw_steps']}",
          file=sys.stderr, flush=True)
    return out


def vertex_sampling(P, t, g, flush, ratios=(0.1, 0.3, 0.5, 0.7, 0.9, 1.0), steps=10):
    """Section 9's scalability experiment on this graph: a share `ratio` of
    the vertices is sampled (a fixed uniform draw per vertex), the others are
    DEAD from the start (trim_set_dead_mask); each fixed variant is timed."""
    u = np.random.default_rng(2024).random(g.n)
    out = {}
    for ratio in ratios:
        t.set_dead_mask((u >= ratio).astype(np.uint8))
        row = {"sampled_vertices": int((u < ratio).sum())}
        for v in ("ac4", "ac6", "ac3"):
            ts, ks, st = time_variant(P, t, v, steps, 1, flush)
            row[v] = {"ms": statistics.mean(ts), "rounds": st["rounds"], "trimmed": st["n_dead"]}
        out[f"{ratio:.1f}"] = row
        print(f"# sampled {ratio:.1f}: " + "  ".join(f"{v} {row[v]['ms']:.4f} ms"
                                                   for v in ("ac4", "ac6", "ac3"))
              + f"  trimmed {row['ac4']['trimmed']}", file=sys.stderr, flush=True)
    t.set_dead_mask(None)
    return out


def implicit_comparison(P, flush, stream, steps=3):
    """Section 2.1's on-the-fly property: the deep-cascade recipe (2^24
    vertices, chains) as an implicit graph whose successors the AC-6 and AC-3
    kernels compute, against the same graph stored as a CSR (configs index 2).
    Reports time and edges inspected (the work counter) for each."""
    import torch
    import graphgen.configs as cfg
    n = 1 << 24
    nC, nR = n // 10, n // 5
    spec = dict(seed=3, nC=nC, nR=nR, nT=n - nC - nR, c_k=(8, 8), r_k=(1, 15), t_k=(0, 14),
                n_chains=4096)
    out = {"workload": "deep_cascade recipe (2^24 vertices, 4,096 chains), seed 3: implicit "
                       "(successors computed by the kernels) and stored as a CSR"}
    g = cfg.config(2)
    oi, ti = host_transpose(g.off, g.tgt)
    dev = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    for kind in ("implicit", "csr"):
        make = (lambda flags=0: P.Trimmer.implicit(**spec, stream=stream, flags=flags)) \
            if kind == "implicit" else \
            (lambda flags=0: P.Trimmer(dev(g.off), dev(g.tgt), dev(oi), dev(ti), stream=stream,
                                       flags=flags))
        row = {}
        for v in ("ac6", "ac3"):
            with make(P.TRIM_FLAG_STATS) as t:
                inspected = t.run(v)["edges_inspected"]
            with make() as t:
                ts, ks, st = time_variant(P, t, v, steps, 1, flush)
            ms = statistics.mean(ts)
            row[v] = {"ms": ms, "edges_inspected": int(inspected),
                      "inspected_per_s": inspected / (ms * 1e-3), "rounds": st["rounds"]}
            print(f"# {kind:8s} {v}: {ms:9.3f} ms  inspected {inspected:.3e}", file=sys.stderr,
                  flush=True)
        out[kind] = row
    out["m_csr"] = g.m
    return out


def gt_build_ms(P, bufs, flush, stream, reps=3):
    """Device-side G^T build on a context given only the out-CSR (device
    arrays): CUDA events on the library stream around the first AC-4 run, which
    builds G^T before its launch, minus the same run on the built G^T; median
    over `reps` fresh contexts."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(t):
        flush.add_(1)
        e0.record(stream)
        t.run_async("ac4")
        e1.record(stream)
        t.sync()
        e1.synchronize()
        return e0.elapsed_time(e1)

    out = []
    for _ in range(reps):
        with P.Trimmer(bufs[0], bufs[1], stream=stream) as t:
            first = timed(t)
            out.append(first - statistics.median(timed(t) for _ in range(3)))
    return statistics.median(out)


def extra_workload(P, idx, args, flush, stream, model):
    """A second workload timed in the same run (all its schedules; for the
    batched workload also each graph trimmed alone), as a sub-object of the
    JSON line."""
    import torch
    g, wname = workload(idx)
    oi, ti = host_transpose(g.off, g.tgt)
    dev = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    bufs = [dev(g.off), dev(g.tgt), dev(oi), dev(ti)]
    batched = idx == 3
    gofs = g.graph_off if batched else None
    names = ["ac4", "ac6", "ac3", "heuristic"] + (["learned"] if model is not None else []) \
        + ([] if batched else ["inout"])
    sampling = None
    with P.Trimmer(*bufs, stream=stream) as t:
        if model is not None:
            t.set_model(model)
        sweep = sweep_variants(P, t, g, args, tuned_key(idx, False), names, flush, gofs,
                               label=f"[{idx}] ")
        if idx == 1:
            sampling = vertex_sampling(P, t, g, flush)
        scc = scc_timing(t, g)
    gt_ms = gt_build_ms(P, bufs, flush, stream) if not batched else None
    out = {"workload": wname, "n": g.n, "m": g.m, "variants": sweep,
           "schedules": schedules_summary(sweep)}
    if sampling:
        out["vertex_sampling"] = sampling
    out["scc"] = scc
    if gt_ms is not None:
        out["gt_build_ms"] = gt_ms
        print(f"# [{idx}] device G^T build {gt_ms:.3f} ms", file=sys.stderr, flush=True)
    if batched:
        out["graphs"] = int(len(g.graph_off) - 1)
        out["timing"] = ("CUDA events around trim_batch_run: one replayed CUDA graph "
                         "(control-block reset + persistent kernel) for all graphs")
        ms, cnt = per_graph_fixed(P, g, "ac4", args.per_graph if args.per_graph > 0 else None)
        best = min(sweep[v]["ms"] for v in ("ac4", "ac6", "ac3"))
        out["split_by_size"] = split_by_size(P, g, args, flush, stream)
        out["per_graph_fixed"] = {"schedule": "ac4, each graph trimmed alone (one launch each)",
                                  "ms": ms, "value": g.m / (ms * 1e-3), "unit": UNIT,
                                  "graphs_timed": cnt, "batched_speedup": ms / best}
    del bufs
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, ws, local):
    import torch
    import paper_2107_12720_gb300 as P
    torch.cuda.set_device(local)
    g, wname = workload(args.config, args.small)
    off_in, tgt_in = host_transpose(g.off, g.tgt)
    dev = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    d_off, d_tgt, d_oi, d_ti = dev(g.off), dev(g.tgt), dev(off_in), dev(tgt_in)
    flush = torch.empty(256 << 20 >> 2, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    # timed runs carry no instrumentation; one extra run of a context with
    # TRIM_FLAG_STATS afterwards supplies the work counters
    t = P.Trimmer(d_off, d_tgt, d_oi, d_ti, stream=stream)
    model_path = os.path.join(ROOT, "paper_2107_12720_gb300", "models", "scheduler_mlp.npy")
    model = np.load(model_path) if os.path.exists(model_path) else None
    if model is not None:
        t.set_model(model)
    # the plain variants are the measured schedules of the single-graph
    # workloads; the large mixed graph runs the learned scheduler
    headline = args.variant or ("learned" if (args.config == 4 and model is not None) else "ac4")
    # the batched workload is a packed set of independent graphs; the large
    # mixed graph is also a union of parts, but one graph to trim
    batched = g.graph_off is not None and args.config == 3
    gofs = g.graph_off if batched else None
    key = tuned_key(args.config, args.small)

    sweep = {}
    if args.sweep and rank == 0:
        if args.sweep_variants:
            names = args.sweep_variants.split(",")
        else:
            # AC-3 sweeps the live set every round: on the 10,004-round large
            # graph that is hours of work, so it is left out there
            names = (["ac4", "ac6"] + ([] if args.config == 4 and not args.small else ["ac3"])
                     + ["heuristic"] + (["learned"] if model is not None else [])
                     + ([] if batched else ["inout"]))
        sweep = sweep_variants(P, t, g, args, key, names, flush, gofs)

    tuned = apply_tuned(t, args, headline, key)
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    for _ in range(args.warmup):
        t.batch_run(gofs, headline) if batched else t.run(headline)
    barrier(ws)
    torch.cuda.synchronize()
    times_ms, ks, st = time_variant(P, t, headline, args.steps, 0, flush, gofs)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop() if rank == 0 else None
    step_s = statistics.mean(times_ms) * 1e-3
    total_s = max_over_ranks(sum(times_ms) * 1e-3, ws)
    edges_total = sum_over_ranks(float(g.m) * args.steps, ws)
    value = edges_total / total_s
    kernel_ms = statistics.mean(ks)

    counts = st
    if rank == 0:
        with P.Trimmer(d_off, d_tgt, d_oi, d_ti, stream=stream, flags=P.TRIM_FLAG_STATS) as tc:
            if model is not None:
                tc.set_model(model)
            apply_tuned(tc, args, headline, key)
            counts = tc.batch_run(gofs, headline) if batched else tc.run(headline)
    rate, probed = None, 0
    if rank == 0 and counts["in_edges_pushed"] and not args.no_atomic_probe:
        rate, probed = atomic_ceiling(P, t, off_in, tgt_in, counts["in_edges_pushed"])
    t.close()

    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        full = None
        if tuned:
            from paper_2107_12720_gb300 import autotune
            full = {**autotune.default_params(), **tuned}
        ev, copied, d2h = e2e_measure(P, g, off_in, tgt_in, headline, args.e2e_steps, gofs, True,
                                      full, model)
        evc, _, _ = e2e_measure(P, g, off_in, tgt_in, headline, args.e2e_steps, gofs, False,
                                full, model)
        e2e = {"value": ev * ws, "unit": UNIT,
               "h2d_bytes_per_step": touched_input_bytes(g.n, counts),
               "d2h_bytes_per_step": d2h,
               "inputs": "page-locked host CSR + G^T read in place by the kernels "
                         "(TRIM_MEM_HOST_MAPPED, NVLink-C2C); levels copied back to host. "
                         "h2d_bytes_per_step: the distinct CSR entries the kernels read, from "
                         "the work counters (both offset arrays, the G^T row of every pushed "
                         "in-edge, the target of every inspected out-edge)",
               "host_csr_bytes": copied,
               "copy_inputs_value": evc * ws,
               "copy_inputs": f"same calls with the whole CSR + G^T ({copied} bytes) first "
                              "copied to device memory (TRIM_MEM_HOST)"}

    extra = {}
    if rank == 0 and args.extra and args.config == 4 and not args.small:
        for idx in (1, 3):
            extra[f"config{idx}"] = extra_workload(P, idx, args, flush, stream, model)
        extra["implicit"] = implicit_comparison(P, flush, stream)
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(g.n, counts, {})
    achieved = alg / (kernel_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "ms_per_step_ci95": (1.96 * statistics.stdev(times_ms) / len(times_ms) ** 0.5)
        if len(times_ms) > 1 else None,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wname, "n": g.n, "m": g.m, "schedule": headline,
                   "rounds": st["rounds"], "rounds_by_variant": st["rounds_by_variant"],
                   "segments": st["segments"],
                   "async_from_round": st.get("async_round", 0),
                   "async_rebalances": st.get("async_rebalances", 0),
                   "params": tuned or "library defaults",
                   "l2": "flushed before every step (256 MB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "timing": "CUDA events on the library stream around trim_run_async: reset "
                             "+ persistent kernel (a scheduled run: its first kernel + the "
                             "all-variant continuation behind it)"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": st["launches"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic(args.config, args.small, headline),
                     "kernel": "trim_persistent_kernel (all launches of one run)",
                     "kernel_ms": kernel_ms,
                     "algorithmic_bytes": alg, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "l2_atomics": None if rate is None else {
                         "ops": counts["in_edges_pushed"], "ceiling_ops_per_s": rate,
                         "ceiling_ms": counts["in_edges_pushed"] / rate * 1e3,
                         "share_of_kernel_ms": counts["in_edges_pushed"] / rate * 1e3 / kernel_ms,
                         "probe": f"trim_probe_atomic_rate: returning atomicSub on the run's own "
                                  f"counter indices ({probed} of them), one fully parallel kernel"}},
    }
    if sweep:
        line["variants"] = sweep
        line["schedules"] = schedules_summary(sweep)
    if batched:
        line["config"]["graphs"] = int(len(g.graph_off) - 1)
        line["config"]["timing"] = ("CUDA events around trim_batch_run: one replayed CUDA graph "
                                    "(control-block reset + persistent kernel) for all graphs")
        if args.per_graph:
            ms, cnt = per_graph_fixed(P, g, "ac4", None if args.per_graph <= 0 else args.per_graph)
            line["per_graph_fixed"] = {"schedule": "ac4, each graph trimmed alone", "ms": ms,
                                       "value": g.m / (ms * 1e-3), "unit": UNIT,
                                       "graphs_timed": cnt,
                                       "batched_speedup": ms / (step_s * 1e3)}
    if extra:
        line["other_workloads"] = extra
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(g, (off_in, tgt_in), args.cpu_seconds)
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--variant", default=None)
    ap.add_argument("--small", action="store_true",
                    help="the small case of --config (parity-test size), for profiling")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip timing every variant next to the headline schedule")
    ap.add_argument("--sweep-variants", default="", help="comma-separated subset for --sweep")
    ap.add_argument("--sweep-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="large mixed workload: skip timing the R-MAT scale-22 and batched "
                         "workloads beside it")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tuned", action="store_true",
                    help="library default parameters instead of the autotuned ones")
    ap.add_argument("--no-atomic-probe", action="store_true",
                    help="skip measuring the L2 atomic ceiling of the run's pushes")
    ap.add_argument("--per-graph", type=int, default=256,
                    help="batched workload: also time each graph alone (N>0: a sample of N graphs "
                         "scaled to all, -1: all, 0: skip)")
    args = ap.parse_args(argv)
    rank, ws, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

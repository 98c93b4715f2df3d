"""ctypes declarations of include/trim.h and thin wrappers with the same names.

Loading fails loudly (TrimError) if libtrim.so has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrim.so")

TRIM_LIVE = 0xFFFFFFFF
TRIM_MASKED = 0xFFFFFFFE
TRIM_AC4_PUSH, TRIM_AC6_SUPPORT, TRIM_AC3_PULL = 0, 1, 2
TRIM_SCHED_HEURISTIC, TRIM_SCHED_LEARNED, TRIM_SCHED_SCRIPTED = 3, 4, 5
TRIM_FLAG_VALIDATE, TRIM_FLAG_STATS, TRIM_FLAG_ROUND_LOG = 1, 2, 4
TRIM_MEM_HOST, TRIM_MEM_DEVICE, TRIM_MEM_HOST_MAPPED = 0, 1, 2
TRIM_HANDOVER_DEVICE, TRIM_HANDOVER_HOST, TRIM_HANDOVER_NONE = 0, 1, 2
TRIM_MLP_NIN, TRIM_MLP_NH, TRIM_MLP_NOUT = 12, 32, 3
TRIM_MLP_NPARAMS = 1571
TRIM_MLP_NBLOB = TRIM_MLP_NPARAMS + 4 * TRIM_MLP_NIN
ERR_NAMES = {0: "TRIM_OK", 1: "TRIM_ERR_INVALID_ARG", 2: "TRIM_ERR_BAD_GRAPH",
             3: "TRIM_ERR_TOO_LARGE", 4: "TRIM_ERR_OOM", 5: "TRIM_ERR_CUDA",
             6: "TRIM_ERR_TIMEOUT", 7: "TRIM_ERR_STATE", 8: "TRIM_ERR_NO_DEVICE"}


class TrimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class TrimCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64), ("offsets", ctypes.c_void_p),
                ("targets", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class TrimParams(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("sched_commit_rounds", ctypes.c_uint32), ("sched_recheck_rounds", ctypes.c_uint32),
                ("spin_limit_ns", ctypes.c_uint64), ("heur_push_ratio", ctypes.c_float),
                ("heur_ac6_ratio", ctypes.c_float), ("local_round_edges", ctypes.c_uint32),
                ("sched_commit_confidence", ctypes.c_float), ("sched_handover", ctypes.c_uint32),
                ("async_round_edges", ctypes.c_uint32)]


class TrimImplicitGraph(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("salt", ctypes.c_uint64)] + [
        (k, ctypes.c_uint32) for k in ("nC", "nR", "nT", "c_kmin", "c_kmax", "r_kmin", "r_kmax",
                                       "t_sinks", "t_kmin", "t_kmax", "n_chains")]


class TrimSccStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("components", "trimmed_size1", "trimmed_size2",
                                               "trimmed_in_steps", "fwbw_steps",
                                               "search_levels")] + [("ms", ctypes.c_float)]


class TrimRunStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("n_dead", ctypes.c_uint32),
                ("device_ms", ctypes.c_float), ("edges_inspected", ctypes.c_uint64),
                ("in_edges_pushed", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("live_swept", ctypes.c_uint64), ("rounds_by_variant", ctypes.c_uint32 * 3),
                ("segments", ctypes.c_uint32), ("local_rounds", ctypes.c_uint32),
                ("launches", ctypes.c_uint32), ("async_round", ctypes.c_uint32),
                ("async_removed", ctypes.c_uint32), ("async_rebalances", ctypes.c_uint32)]


class TrimRoundRec(ctypes.Structure):
    _fields_ = [("round", ctypes.c_uint32), ("variant", ctypes.c_uint32),
                ("frontier", ctypes.c_uint32), ("removed", ctypes.c_uint32),
                ("t_start_ns", ctypes.c_uint64), ("t_end_ns", ctypes.c_uint64),
                ("t_work_ns", ctypes.c_uint64), ("t_flush_ns", ctypes.c_uint64),
                ("features", ctypes.c_float * 12)]


# every symbol declared in include/trim.h: (name, restype, argtypes)
_P = ctypes.c_void_p
_U32, _U64, _F, _SZ, _I = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t, ctypes.c_int
SIGNATURES = [
    ("trim_create", _I, [ctypes.POINTER(TrimCsr), ctypes.POINTER(TrimCsr), _P, _U32,
                         ctypes.POINTER(_P)]),
    ("trim_run", _I, [_P, _I, ctypes.POINTER(TrimRunStats)]),
    ("trim_run_inout", _I, [_P, ctypes.POINTER(TrimRunStats)]),
    ("trim_run_scc", _I, [_P, _P, _I, ctypes.POINTER(TrimSccStats)]),
    ("trim_create_implicit", _I, [ctypes.POINTER(TrimImplicitGraph), _P, _U32,
                                  ctypes.POINTER(_P)]),
    ("trim_set_dead_mask", _I, [_P, _P, _I]),
    ("trim_run_async", _I, [_P, _I]),
    ("trim_sync", _I, [_P, ctypes.POINTER(TrimRunStats)]),
    ("trim_status", _I, [_P, _P, _I]),
    ("trim_level", _I, [_P, _P, _I]),
    ("trim_level_device_ptr", _I, [_P, ctypes.POINTER(_P)]),
    ("trim_in_csr", _I, [_P, _P, _P, _I]),
    ("trim_batch_run", _I, [_P, _P, _U32, _I, ctypes.POINTER(TrimRunStats)]),
    ("trim_set_params", _I, [_P, ctypes.POINTER(TrimParams)]),
    ("trim_get_params", _I, [_P, ctypes.POINTER(TrimParams)]),
    ("trim_default_params", _I, [ctypes.POINTER(TrimParams)]),
    ("trim_set_model", _I, [_P, _P, _SZ]),
    ("trim_set_schedule", _I, [_P, _P, _U32]),
    ("trim_get_round_log", _I, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    ("trim_destroy", None, [_P]),
    ("trim_set_alloc_limit", _I, [_U64]),
    ("trim_last_error", ctypes.c_char_p, [_P]),
    ("trim_mlp_scratch_bytes", _SZ, [_U32]),
    ("trim_mlp_forward", _I, [_P, _P, _U32, _P, _P]),
    ("trim_mlp_loss_grad", _I, [_P, _P, _P, _U32, _P, _P, _P, _P]),
    ("trim_mlp_adam_step", _I, [_P, _P, _P, _P, _U32, _F, _F, _F, _F, _P]),
    ("trim_run_ac4_noalloc", _I, [_P, _P, _P, _P, _U32, _U32, _P, ctypes.POINTER(_U32), _P]),
    ("trim_probe_atomic_rate", _I, [_P, ctypes.c_uint64, _P, _U32, _U32, _P,
                                    ctypes.POINTER(ctypes.c_float)]),
]

_lib = None


def lib():
    """The loaded libtrim.so (raises TrimError if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TrimError(5, f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2107_12720_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code: int, ctx=None) -> None:
    if code != 0:
        msg = lib().trim_last_error(ctx)
        raise TrimError(code, msg.decode() if msg else "")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def trim_create(csr_out: TrimCsr, csr_in, stream, flags: int):
    ctx = ctypes.c_void_p()
    rc = lib().trim_create(ctypes.byref(csr_out), ctypes.byref(csr_in) if csr_in else None,
                           stream, flags, ctypes.byref(ctx))
    check(rc, None)
    return ctx


def trim_run(ctx, variant: int) -> TrimRunStats:
    s = TrimRunStats()
    check(lib().trim_run(ctx, variant, ctypes.byref(s)), ctx)
    return s


def trim_create_implicit(graph: TrimImplicitGraph, stream, flags: int):
    ctx = ctypes.c_void_p()
    check(lib().trim_create_implicit(ctypes.byref(graph), stream, flags, ctypes.byref(ctx)), None)
    return ctx


def trim_run_scc(ctx, comp, out_on_device: int) -> TrimSccStats:
    s = TrimSccStats()
    check(lib().trim_run_scc(ctx, _ptr(comp), out_on_device, ctypes.byref(s)), ctx)
    return s


def trim_run_inout(ctx) -> TrimRunStats:
    s = TrimRunStats()
    check(lib().trim_run_inout(ctx, ctypes.byref(s)), ctx)
    return s


def trim_set_dead_mask(ctx, mask, on_device: int) -> None:
    check(lib().trim_set_dead_mask(ctx, _ptr(mask), on_device), ctx)


def trim_run_async(ctx, variant: int) -> None:
    check(lib().trim_run_async(ctx, variant), ctx)


def trim_sync(ctx) -> TrimRunStats:
    s = TrimRunStats()
    check(lib().trim_sync(ctx, ctypes.byref(s)), ctx)
    return s


def trim_status(ctx, out_ptr, on_device: int) -> None:
    check(lib().trim_status(ctx, _ptr(out_ptr), on_device), ctx)


def trim_level(ctx, out_ptr, on_device: int) -> None:
    check(lib().trim_level(ctx, _ptr(out_ptr), on_device), ctx)


def trim_in_csr(ctx, off_ptr, tgt_ptr, on_device: int) -> None:
    check(lib().trim_in_csr(ctx, _ptr(off_ptr), _ptr(tgt_ptr), on_device), ctx)


def trim_level_device_ptr(ctx) -> int:
    p = ctypes.c_void_p()
    check(lib().trim_level_device_ptr(ctx, ctypes.byref(p)), ctx)
    return p.value


def trim_batch_run(ctx, graph_off: np.ndarray, variant: int) -> TrimRunStats:
    go = np.ascontiguousarray(graph_off, np.uint32)
    s = TrimRunStats()
    check(lib().trim_batch_run(ctx, go.ctypes.data, go.shape[0] - 1, variant, ctypes.byref(s)),
          ctx)
    return s


def trim_default_params() -> TrimParams:
    p = TrimParams()
    check(lib().trim_default_params(ctypes.byref(p)))
    return p


def trim_get_params(ctx) -> TrimParams:
    p = TrimParams()
    check(lib().trim_get_params(ctx, ctypes.byref(p)), ctx)
    return p


def trim_set_params(ctx, p: TrimParams) -> None:
    check(lib().trim_set_params(ctx, ctypes.byref(p)), ctx)


def trim_set_model(ctx, blob) -> None:
    if blob is None:
        check(lib().trim_set_model(ctx, None, 0), ctx)
    else:
        b = np.ascontiguousarray(blob, np.float32)
        check(lib().trim_set_model(ctx, b.ctypes.data, b.size), ctx)


def trim_set_schedule(ctx, variants) -> None:
    v = np.ascontiguousarray(variants, np.uint8)
    check(lib().trim_set_schedule(ctx, v.ctypes.data if v.size else None, v.size), ctx)


def trim_get_round_log(ctx, cap: int = 1 << 20):
    buf = (TrimRoundRec * cap)()
    n = ctypes.c_size_t(0)
    check(lib().trim_get_round_log(ctx, buf, cap, ctypes.byref(n)), ctx)
    return list(buf[: n.value])


def trim_destroy(ctx) -> None:
    lib().trim_destroy(ctx)


def trim_last_error(ctx=None) -> str:
    return lib().trim_last_error(ctx).decode()


def trim_set_alloc_limit(nbytes: int) -> None:
    check(lib().trim_set_alloc_limit(nbytes))


def trim_mlp_scratch_bytes(N: int) -> int:
    return int(lib().trim_mlp_scratch_bytes(N))


def trim_mlp_forward(params, X, N: int, logits, stream) -> None:
    check(lib().trim_mlp_forward(_ptr(params), _ptr(X), N, _ptr(logits), stream))


def trim_mlp_loss_grad(params, X, y, N: int, loss, grad, scratch, stream) -> None:
    check(lib().trim_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(y), N, _ptr(loss), _ptr(grad),
                                   _ptr(scratch), stream))


def trim_mlp_adam_step(params, grad, m, v, t: int, lr: float, beta1: float, beta2: float,
                       eps: float, stream) -> None:
    check(lib().trim_mlp_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), t, lr, beta1,
                                   beta2, eps, stream))


TRIM_NOALLOC_MAX_N = 1 << 18
TRIM_NOALLOC_MAX_M = 1 << 22


def trim_run_ac4_noalloc(offsets, targets, in_offsets, in_targets, n: int, m: int, level_out,
                         stream) -> int:
    """AC-4 trimming with the library's fixed scratch array (no device allocation);
    all arrays are device tensors/pointers. Returns alpha."""
    rounds = ctypes.c_uint32(0)
    rc = lib().trim_run_ac4_noalloc(_ptr(offsets), _ptr(targets), _ptr(in_offsets),
                                    _ptr(in_targets), n, m, _ptr(level_out),
                                    ctypes.byref(rounds), stream)
    if rc != 0:
        raise TrimError(rc, "trim_run_ac4_noalloc failed")
    return int(rounds.value)


def trim_probe_atomic_rate(idx, n_idx: int, counters, n_counters: int, reps: int, stream) -> float:
    """Fastest of `reps` fully parallel passes of returning atomicSub over the
    counter indices idx (device); counters (device) is overwritten. Returns ms."""
    ms = ctypes.c_float(0.0)
    check(lib().trim_probe_atomic_rate(_ptr(idx), n_idx, _ptr(counters), n_counters, reps, stream,
                                       ctypes.byref(ms)), None)
    return float(ms.value)

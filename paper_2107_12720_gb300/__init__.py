"""Python binding of the GB300 graph-trimming library (include/trim.h).

Argument marshalling only: every step of the trimming runs in the CUDA kernels
of ``libtrim.so``. There is no CPU fallback; if the library is missing or no
sm_103 device is present, calls raise ``TrimError``.

Low-level functions carry the C names (``trim_create``, ``trim_run``,
``trim_status``, ``trim_level``, ``trim_batch_run``, ...). ``Trimmer`` wraps a
context for use with torch tensors (device memory and streams come from torch).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .abi import (LIB_PATH, TRIM_MASKED, TRIM_AC3_PULL, TRIM_AC4_PUSH, TRIM_AC6_SUPPORT, TRIM_FLAG_ROUND_LOG,
                  TRIM_FLAG_STATS, TRIM_FLAG_VALIDATE, TRIM_LIVE, TRIM_MEM_DEVICE, TRIM_MEM_HOST,
                  TRIM_MEM_HOST_MAPPED, TRIM_MLP_NBLOB, TRIM_HANDOVER_DEVICE, TRIM_HANDOVER_HOST,
                  TRIM_HANDOVER_NONE,
                  TRIM_MLP_NPARAMS, TRIM_SCHED_HEURISTIC, TRIM_SCHED_LEARNED,
                  TRIM_SCHED_SCRIPTED, TrimCsr, TrimError, TrimImplicitGraph, TrimParams,
                  TrimRoundRec,
                  TrimRunStats, lib, check)
from .abi import (trim_batch_run, trim_create, trim_create_implicit, trim_default_params,
                  trim_destroy,
                  trim_get_params, trim_get_round_log, trim_last_error, trim_level,
                  trim_level_device_ptr, trim_in_csr, trim_mlp_adam_step, trim_mlp_forward, trim_mlp_loss_grad,
                  trim_mlp_scratch_bytes, trim_run, trim_run_async, trim_run_inout, trim_run_scc,
                  trim_set_alloc_limit, trim_set_dead_mask,
                  trim_set_model, trim_set_params, trim_set_schedule, trim_status, trim_sync)

VARIANTS = {"ac4": TRIM_AC4_PUSH, "ac6": TRIM_AC6_SUPPORT, "ac3": TRIM_AC3_PULL,
            "heuristic": TRIM_SCHED_HEURISTIC, "learned": TRIM_SCHED_LEARNED,
            "scripted": TRIM_SCHED_SCRIPTED}

__all__ = ["Trimmer", "TrimError", "VARIANTS", "lib", "LIB_PATH"]


def _as_u32(a) -> np.ndarray:
    """A uint32 view of a 32-bit integer array (no copy: a pinned host buffer
    stays pinned); other dtypes or layouts are converted."""
    a = np.asarray(a)
    if a.dtype in (np.int32, np.uint32) and a.flags.c_contiguous:
        return a.view(np.uint32)
    return np.ascontiguousarray(a, np.uint32)


def _variant(v) -> int:
    if isinstance(v, str):
        return VARIANTS[v]
    return int(v)


class Trimmer:
    """One trimming context over a CSR graph.

    ``off``/``tgt`` (and optionally ``off_in``/``tgt_in`` for G^T) are uint32
    arrays: CUDA torch tensors are borrowed (kept alive by this object), numpy
    arrays or CPU tensors are copied to the device by the library, or, with
    ``host_mapped=True``, read in place by the kernels (TRIM_MEM_HOST_MAPPED:
    page-locked memory such as ``tensor.pin_memory()``, or any host memory on a
    GPU that reads pageable memory; kept alive by this object).
    """

    def __init__(self, off, tgt, off_in=None, tgt_in=None, stream=None, flags: int = 0,
                 host_mapped: bool = False):
        import torch
        self._keep = []
        self._host_mode = TRIM_MEM_HOST_MAPPED if host_mapped else TRIM_MEM_HOST
        out_csr = self._csr(off, tgt)
        in_csr = self._csr(off_in, tgt_in) if off_in is not None else None
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        self.ctx = trim_create(out_csr, in_csr, sp, flags)
        self.n = out_csr.n
        self.m = out_csr.m
        self.flags = flags

    @classmethod
    def implicit(cls, seed: int, nC: int, nR: int, nT: int, c_k=(4, 4), r_k=(1, 4), t_sinks=0,
                 t_k=(1, 4), n_chains=0, salt: int = 0, stream=None, flags: int = 0):
        """A context over the library's implicit planted graph (no CSR in
        memory; successors computed on the fly, see trim_create_implicit).
        Only run("ac6") and run("ac3") apply."""
        import torch
        self = cls.__new__(cls)
        self._keep = []
        g = TrimImplicitGraph(seed, salt, nC, nR, nT, c_k[0], c_k[1], r_k[0], r_k[1], t_sinks,
                              t_k[0], t_k[1], n_chains)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        self.ctx = trim_create_implicit(g, sp, flags)
        self.n = nC + nR + nT
        self.m = None
        self.flags = flags
        return self

    def _csr(self, off, tgt):
        import torch
        if isinstance(off, torch.Tensor) and off.is_cuda:
            off = off.contiguous()
            tgt = tgt.contiguous()
            if off.dtype not in (torch.int32, torch.uint32) or tgt.dtype not in (torch.int32,
                                                                                   torch.uint32):
                raise TrimError(1, "CSR tensors must be 32-bit integers")
            self._keep += [off, tgt]
            return TrimCsr(off.numel() - 1, tgt.numel(), off.data_ptr(),
                           tgt.data_ptr() if tgt.numel() else None, TRIM_MEM_DEVICE)
        if isinstance(off, torch.Tensor):
            self._keep += [off, tgt]  # a pinned tensor must outlive a mapped context
            off = off.numpy()
            tgt = tgt.numpy()
        off, tgt = _as_u32(off), _as_u32(tgt)
        self._keep += [off, tgt]
        return TrimCsr(off.shape[0] - 1, tgt.shape[0], off.ctypes.data,
                       tgt.ctypes.data if tgt.size else None, self._host_mode)

    def run(self, variant="ac4") -> dict:
        return _stats_dict(trim_run(self.ctx, _variant(variant)))

    def set_dead_mask(self, mask) -> None:
        """Vertices with mask != 0 are DEAD from the start of every later run
        (vertex sampling); None clears the mask. numpy / CPU tensor: host,
        CUDA tensor: device (copied either way)."""
        import torch
        if mask is None:
            trim_set_dead_mask(self.ctx, None, 0)
            return
        if isinstance(mask, torch.Tensor) and mask.is_cuda:
            if mask.numel() != self.n:
                raise TrimError(1, "mask must have n entries")
            m = (mask != 0).to(torch.uint8).contiguous()
            trim_set_dead_mask(self.ctx, m.data_ptr(), 1)
            return
        m = np.ascontiguousarray(np.asarray(mask) != 0, np.uint8)
        if m.shape[0] != self.n:
            raise TrimError(1, "mask must have n entries")
        trim_set_dead_mask(self.ctx, m.ctypes.data, 0)

    def run_scc(self, device: bool = False):
        """SCC decomposition (trim_run_scc): returns (comp, stats) with comp[v]
        the smallest vertex id of v's strongly connected component."""
        import torch
        if device:
            comp = torch.empty(self.n, dtype=torch.int32, device="cuda")
            s = trim_run_scc(self.ctx, comp.data_ptr(), 1)
        else:
            comp = np.empty(self.n, np.uint32)
            s = trim_run_scc(self.ctx, comp.ctypes.data, 0)
        return comp, {k: getattr(s, k) for k, _ in s._fields_}

    def run_inout(self) -> dict:
        """In+out trimming (no live successor or no live predecessor removes a
        vertex); results through level() and status() as after run()."""
        return _stats_dict(trim_run_inout(self.ctx))

    def run_async(self, variant="ac4") -> None:
        trim_run_async(self.ctx, _variant(variant))

    def sync(self) -> dict:
        return _stats_dict(trim_sync(self.ctx))

    def batch_run(self, graph_off, variant="ac4") -> dict:
        go = np.ascontiguousarray(graph_off, np.uint32)
        return _stats_dict(trim_batch_run(self.ctx, go, _variant(variant)))

    def level(self, device: bool = True):
        import torch
        if device:
            out = torch.empty(self.n, dtype=torch.int32, device="cuda")
            trim_level(self.ctx, out.data_ptr(), 1)
            return out.view(torch.uint32) if hasattr(torch, "uint32") else out
        out = np.empty(self.n, np.uint32)
        trim_level(self.ctx, out.ctypes.data, 0)
        return out

    def in_csr(self):
        """G^T as host arrays (in_offsets, in_targets); built on the device
        first if the context was created without it (see trim_in_csr)."""
        off = np.empty(self.n + 1, np.uint32)
        tgt = np.empty(max(int(self.m), 1), np.uint32)
        trim_in_csr(self.ctx, off.ctypes.data, tgt.ctypes.data, 0)
        return off, tgt[:int(self.m)]

    def status(self, device: bool = True):
        import torch
        if device:
            out = torch.empty(self.n, dtype=torch.uint8, device="cuda")
            trim_status(self.ctx, out.data_ptr(), 1)
            return out
        out = np.empty(self.n, np.uint8)
        trim_status(self.ctx, out.ctypes.data, 0)
        return out

    def set_params(self, **kw) -> None:
        p = trim_get_params(self.ctx)
        for k, v in kw.items():
            setattr(p, k, v)
        trim_set_params(self.ctx, p)

    def params(self) -> dict:
        p = trim_get_params(self.ctx)
        return {k: getattr(p, k) for k, _ in TrimParams._fields_}

    def set_model(self, blob) -> None:
        trim_set_model(self.ctx, None if blob is None else np.ascontiguousarray(blob, np.float32))

    def set_schedule(self, variants) -> None:
        trim_set_schedule(self.ctx, np.ascontiguousarray(variants, np.uint8))

    def round_log(self):
        return trim_get_round_log(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            trim_destroy(self.ctx)
            self.ctx = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _stats_dict(s: TrimRunStats) -> dict:
    return {"rounds": s.rounds, "n_dead": s.n_dead, "device_ms": s.device_ms,
            "edges_inspected": s.edges_inspected, "in_edges_pushed": s.in_edges_pushed,
            "candidates": s.candidates, "live_swept": s.live_swept,
            "rounds_by_variant": list(s.rounds_by_variant), "segments": s.segments,
            "local_rounds": s.local_rounds, "launches": s.launches,
            "async_round": s.async_round, "async_removed": s.async_removed,
            "async_rebalances": s.async_rebalances}

"""GB300 reverse k-ranks: exact and c-approximate queries behind a C ABI.

Thin ctypes binding over ``librkr.so`` (built from ``csrc/`` for sm_103a by
``buildlib.build()``).  Functions carry the names of the C entry points
(``rkr_build``, ``rkr_query_exact``, ``rkr_query_approx``); they only marshal
arguments.  Every step of the computation runs in the library's CUDA kernels:
there is no CPU fallback, and using this package without the built library
raises ``RuntimeError``.

Arrays may be numpy arrays (host memory) or torch CUDA tensors (device memory);
the library detects which.  Outputs are numpy arrays unless ``device=True``.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import buildlib

__all__ = ["RKRError", "Index", "QueryStats", "load", "rkr_build", "rkr_query_exact",
           "rkr_query_approx", "rkr_query_exact_subsets", "rkr_query_approx_subsets",
           "rkr_query_approx_single", "rkr_query_approx_candidates", "rkr_merge_approx",
           "rkr_merge_exact",
           "rkr_screen_scores", "rkr_screen_scores_static",
           "rkr_profile_start", "rkr_profile_stop", "Pruner", "rkr_rank_pairs",
           "rkr_pair_features", "rkr_query_exact_learned", "rkr_release_cached_memory",
           "rkr_set_wait_limit", "device_allocations", "version", "EXPORTS", "Tuning",
           "rkr_tuning_get", "rkr_tuning_set", "rkr_autotune", "Session"]

_lock = threading.Lock()
_lib = None

EXPORTS = dict(perm=1, fmin=2, fmax=3, table=4, samples=5, xlo=6, xgrid=7, pnorm=8, xhi=9,
               dlo=10, dhi=11, dgrid=12)
DEEP_GRID = 64   # points of the deep count grid (RKR_DEEP_GRID)
_STATUS = {0: "RKR_OK", 1: "RKR_EINVAL", 2: "RKR_ENOMEM", 3: "RKR_ECUDA", 4: "RKR_ETIMEOUT",
           5: "RKR_EUNSUPPORTED", 6: "RKR_EINTERNAL"}


class RKRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _BuildParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int32), ("omega", ctypes.c_int32), ("s", ctypes.c_int32),
                ("fbounds", ctypes.c_int32), ("exact_table", ctypes.c_int32),
                ("floor_rank", ctypes.c_int32), ("sample_pos", ctypes.c_void_p),
                ("seed", ctypes.c_uint64)]


class QueryStats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("fp64_dots", ctypes.c_int64), ("near_ties", ctypes.c_int64),
                ("wide_queries", ctypes.c_int32), ("max_rel_screen_err", ctypes.c_double),
                ("ms_theta", ctypes.c_double), ("ms_resolve", ctypes.c_double),
                ("ms_select", ctypes.c_double), ("recounted", ctypes.c_int64),
                ("deep_queries", ctypes.c_int32), ("recount_users", ctypes.c_int64),
                ("recount_open", ctypes.c_int64), ("recount_split", ctypes.c_int64),
                ("learned_revived", ctypes.c_int64), ("max_screen_err_ratio", ctypes.c_double),
                ("prefix_rows", ctypes.c_int64), ("prefix_pruned", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tuning(ctypes.Structure):
    """Launch choices that change speed, never results (rkr_tuning)."""
    _fields_ = [("rc_bn", ctypes.c_int32), ("rc_single_first", ctypes.c_int32),
                ("skip_level", ctypes.c_int32), ("cand_budget_log2", ctypes.c_int32),
                ("latency_ctas_per_sm", ctypes.c_int32), ("latency_bulk", ctypes.c_int32),
                ("screen_form", ctypes.c_int32), ("rc_seg_min", ctypes.c_int32),
                ("split_cat", ctypes.c_int32), ("rc_prefix", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def load() -> ctypes.CDLL:
    """Load the library build this process uses (``buildlib.selected_variant()``:
    librkr.so, or librkr_replica.so with RKR_LIB_VARIANT=replica); raises
    RuntimeError when it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = buildlib.lib_path(buildlib.selected_variant())
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "paper_2504_13446_gb300.buildlib.build()")
        lib = ctypes.CDLL(path)
        V, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.rkr_build.restype = I32
        lib.rkr_build.argtypes = [V, I64, V, I64, I32, ctypes.POINTER(_BuildParams), V,
                                  ctypes.POINTER(V)]
        lib.rkr_query_exact.restype = I32
        lib.rkr_query_exact.argtypes = [V, V, I32, V, V, V, ctypes.POINTER(QueryStats), V]
        lib.rkr_query_approx.restype = I32
        lib.rkr_query_approx.argtypes = [V, V, I32, V, ctypes.c_double, V, V, V, V, V, V,
                                         ctypes.POINTER(QueryStats), V]
        lib.rkr_query_exact_subsets.restype = I32
        lib.rkr_query_exact_subsets.argtypes = [V, V, I32, V, V, V, V, V,
                                                ctypes.POINTER(QueryStats), V]
        lib.rkr_session_create.restype = I32
        lib.rkr_session_create.argtypes = [V, I32, ctypes.c_double, V, ctypes.POINTER(V)]
        lib.rkr_session_query.restype = I32
        lib.rkr_session_query.argtypes = [V, V, I32, V, V, V, V, V, V]
        lib.rkr_session_free.restype = None
        lib.rkr_session_free.argtypes = [V]
        lib.rkr_query_exact_bitmap.restype = I32
        lib.rkr_query_exact_bitmap.argtypes = [V, V, I32, V, V, I64, V, V,
                                               ctypes.POINTER(QueryStats), V]
        lib.rkr_query_approx_bitmap.restype = I32
        lib.rkr_query_approx_bitmap.argtypes = [V, V, I32, V, V, I64, ctypes.c_double, V, V, V,
                                                V, V, V, ctypes.POINTER(QueryStats), V]
        lib.rkr_query_approx_single.restype = I32
        lib.rkr_query_approx_single.argtypes = [V, V, I32, V, ctypes.c_double, V, V, V, V, V, V,
                                                ctypes.POINTER(QueryStats), V]
        lib.rkr_query_approx_candidates.restype = I32
        lib.rkr_query_approx_candidates.argtypes = [V, V, I32, V, I64, I64, V, V, V, V, V, V]
        lib.rkr_merge_approx.restype = I32
        lib.rkr_merge_approx.argtypes = [I32, V, ctypes.c_double, I32, V, V, V, V, V, V, V, V,
                                         V, V, V]
        lib.rkr_merge_exact.restype = I32
        lib.rkr_merge_exact.argtypes = [I32, V, V, V, V, V, V]
        lib.rkr_query_approx_subsets.restype = I32
        lib.rkr_query_approx_subsets.argtypes = [V, V, I32, V, V, V, ctypes.c_double, V, V, V,
                                                 V, V, V, ctypes.POINTER(QueryStats), V]
        lib.rkr_index_export.restype = I32
        lib.rkr_index_export.argtypes = [V, I32, V, I64]
        lib.rkr_index_info.restype = I32
        lib.rkr_index_info.argtypes = [V, ctypes.POINTER(I64)]
        lib.rkr_index_free.restype = None
        lib.rkr_index_free.argtypes = [V]
        lib.rkr_index_timings.restype = I32
        lib.rkr_index_timings.argtypes = [V, ctypes.POINTER(ctypes.c_double), I32]
        lib.rkr_kernel_launches.restype = ctypes.c_uint64
        lib.rkr_kernel_launches.argtypes = []
        lib.rkr_release_cached_memory.restype = ctypes.c_int32
        lib.rkr_release_cached_memory.argtypes = []
        lib.rkr_screen_scores.restype = I32
        lib.rkr_screen_scores.argtypes = [V, I64, V, I64, I32, I32, V, V, V]
        lib.rkr_pruner_create.restype = I32
        lib.rkr_pruner_create.argtypes = [I32, I32, ctypes.c_uint64, ctypes.POINTER(V)]
        lib.rkr_pruner_nparams.restype = I64
        lib.rkr_pruner_nparams.argtypes = [V]
        lib.rkr_pruner_params.restype = I32
        lib.rkr_pruner_params.argtypes = [V, I32, V, I64]
        lib.rkr_pruner_forward.restype = I32
        lib.rkr_pruner_forward.argtypes = [V, V, V, I64, V, V]
        lib.rkr_pruner_loss_grads.restype = I32
        lib.rkr_pruner_loss_grads.argtypes = [V, V, V, V, I64, ctypes.POINTER(ctypes.c_float), V, V]
        lib.rkr_pruner_train.restype = I32
        lib.rkr_pruner_train.argtypes = [V, V, V, V, I64, I32, I32, ctypes.c_float,
                                         ctypes.c_uint64, ctypes.POINTER(ctypes.c_float), V]
        lib.rkr_rank_pairs.restype = I32
        lib.rkr_rank_pairs.argtypes = [V, V, I32, I64, V, V, V, V]
        lib.rkr_pair_features.restype = I32
        lib.rkr_pair_features.argtypes = [V, V, V, I32, I64, V, V, V, V, V]
        lib.rkr_query_exact_learned.restype = I32
        lib.rkr_query_exact_learned.argtypes = [V, V, V, V, I32, V, V, I32, V, V,
                                                ctypes.POINTER(QueryStats), V]
        lib.rkr_pruner_invert.restype = I32
        lib.rkr_pruner_invert.argtypes = [V, V, V, I32, V]
        lib.rkr_pruner_table.restype = I32
        lib.rkr_pruner_table.argtypes = [V, I64, I32, V, V]
        lib.rkr_pruner_free.restype = None
        lib.rkr_pruner_free.argtypes = [V]
        lib.rkr_profile_start.restype = I32
        lib.rkr_profile_start.argtypes = []
        lib.rkr_profile_stop.restype = I32
        lib.rkr_profile_stop.argtypes = [ctypes.c_char_p, I64]
        lib.rkr_screen_scores_static.restype = I32
        lib.rkr_screen_scores_static.argtypes = [V, I64, V, I64, I32, I32, V, V, V]
        lib.rkr_index_device_bytes.restype = I32
        lib.rkr_index_device_bytes.argtypes = [V, ctypes.POINTER(I64)]
        lib.rkr_index_save.restype = I32
        lib.rkr_index_save.argtypes = [V, ctypes.c_char_p]
        lib.rkr_index_load.restype = I32
        lib.rkr_index_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(V)]
        lib.rkr_pruner_save.restype = I32
        lib.rkr_pruner_save.argtypes = [V, ctypes.c_char_p]
        lib.rkr_pruner_load.restype = I32
        lib.rkr_pruner_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(V)]
        lib.rkr_tuning_get.restype = I32
        lib.rkr_tuning_get.argtypes = [ctypes.POINTER(Tuning)]
        lib.rkr_tuning_set.restype = I32
        lib.rkr_tuning_set.argtypes = [ctypes.POINTER(Tuning)]
        lib.rkr_autotune.restype = I32
        lib.rkr_autotune.argtypes = [V, V, I32, V, ctypes.c_double, I32, ctypes.c_char_p,
                                     ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double), V]
        lib.rkr_device_allocations.restype = ctypes.c_uint64
        lib.rkr_device_allocations.argtypes = []
        lib.rkr_set_wait_limit.restype = I32
        lib.rkr_set_wait_limit.argtypes = [I64]
        lib.rkr_last_error.restype = ctypes.c_char_p
        lib.rkr_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def rkr_profile_start() -> None:
    """Start per-kernel device-time accounting (CUDA events on the launching stream)."""
    _check(load().rkr_profile_start())


def rkr_profile_stop() -> dict:
    """Stop accounting; {kernel: (launches, total_ms, algorithmic work)}."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().rkr_profile_stop(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms, work = line.rsplit(maxsplit=3)
        out[name] = (int(n), float(ms), float(work))
    return out


def kernel_launches() -> int:
    """Kernels launched by librkr.so in this process so far."""
    return int(load().rkr_kernel_launches())


def rkr_tuning_get() -> dict:
    """The process-wide tuning."""
    t = Tuning()
    _check(load().rkr_tuning_get(ctypes.byref(t)))
    return t.as_dict()


def rkr_tuning_set(**fields) -> None:
    """Change tuning fields (the others keep their values)."""
    t = Tuning()
    _check(load().rkr_tuning_get(ctypes.byref(t)))
    for key, v in fields.items():
        setattr(t, key, int(v))
    _check(load().rkr_tuning_set(ctypes.byref(t)))


def rkr_autotune(index, Q, k, *, c: float = 2.0, what: int = 3, cache_path=None, stream=None):
    """Pick the tuning for this workload by timed trials (rkr_autotune): (tuning, ms)."""
    lib = load()
    nq, _ = _shape(Q)
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    pq, kq = _ptr(Q, np.float32)
    t = Tuning()
    ms = ctypes.c_double()
    _check(lib.rkr_autotune(index, pq, nq, kk.ctypes.data, ctypes.c_double(c), int(what),
                            os.fsencode(cache_path) if cache_path else None, ctypes.byref(t),
                            ctypes.byref(ms), _stream(stream)))
    return t.as_dict(), float(ms.value)


def device_allocations() -> int:
    """Device allocations librkr has requested in this process so far."""
    return int(load().rkr_device_allocations())


def rkr_set_wait_limit(rounds: int) -> None:
    """Test hook: try_wait rounds of the screens' epilogue wait (negative = default)."""
    _check(load().rkr_set_wait_limit(int(rounds)))


def version() -> str:
    """The library's version string, naming its build."""
    return load().rkr_version().decode()


def rkr_release_cached_memory() -> None:
    """Return the device memory the library keeps for reuse to the driver."""
    _check(load().rkr_release_cached_memory())


def _check(st: int):
    if st != 0:
        raise RKRError(st, load().rkr_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keepalive) for a numpy array or a contiguous torch tensor."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.int32: torch.int32, np.uint32: torch.int32,
                np.float64: torch.float64}[dtype]
        if x.dtype != want and not (dtype is np.uint32 and x.dtype == torch.int32):
            raise TypeError(f"tensor dtype {x.dtype}, expected {want}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), a


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _empty(shape, dtype, device: bool):
    if device:
        import torch
        tdt = {np.int32: torch.int32, np.uint32: torch.int32, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device="cuda")
    return np.empty(shape, dtype=dtype)


def _shape(x):
    return tuple(x.shape)


def _same_device(*arrays):
    """CUDA tensors among the arguments must be on the current device (the library
    takes a device pointer as memory of the current device)."""
    devs = {a.device.index for a in arrays if _is_torch(a) and a.is_cuda}
    if devs:
        import torch
        cur = torch.cuda.current_device()
        if devs != {cur}:
            raise RKRError(1, f"CUDA tensors must be on the current device cuda:{cur}")


def rkr_build(U, P, *, tau: int = 500, omega: int = 10, s: int = 100, fbounds: str = "exact",
              exact_table=True, floor_rank: int = 0, sample_pos=None, seed: int = 0,
              stream=None) -> ctypes.c_void_p:
    """Pre-processing (Alg. 1); returns an opaque index handle (free with rkr_index_free).

    exact_table: False / 0 none, True / 1 the exact count table, 2 that and the
    deep count grid below the tail lists."""
    lib = load()
    n, d = _shape(U)
    m, d2 = _shape(P)
    if d != d2:
        raise ValueError("U and P must have the same dimension")
    pu, ku = _ptr(U, np.float32)
    pp, kp = _ptr(P, np.float32)
    ps, ks = _ptr(sample_pos, np.int32)
    prm = _BuildParams(tau, omega, s, {"exact": 0, "cs": 1}[fbounds], int(exact_table),
                       floor_rank, ps, seed)
    h = ctypes.c_void_p()
    _check(lib.rkr_build(pu, n, pp, m, d, ctypes.byref(prm), _stream(stream), ctypes.byref(h)))
    return h


def _subsets_csr(subsets, nq):
    """(offsets int64, users int32) from a list of nq per-query user-id arrays."""
    if len(subsets) != nq:
        raise ValueError("one subset per query")
    off = np.zeros(nq + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(s_) for s_ in subsets])
    users = (np.concatenate([np.asarray(s_, dtype=np.int32) for s_ in subsets])
             if off[-1] else np.zeros(1, np.int32))
    return off, np.ascontiguousarray(users)


def _bitmap_ptr(member):
    """(pointer, words, keepalive) of an (nq, words) uint32 bitmap (numpy or torch)."""
    if _is_torch(member):
        if not member.is_contiguous():
            raise ValueError("bitmap tensor must be contiguous")
        return ctypes.c_void_p(member.data_ptr()), int(member.shape[1]), member
    a = np.ascontiguousarray(member, dtype=np.uint32)
    return a.ctypes.data_as(ctypes.c_void_p), int(a.shape[1]), a


def rkr_query_exact(index, Q, k, *, subsets=None, member=None, device: bool = False,
                    stream=None):
    """Exact reverse k-ranks: (users, ranks, offsets, stats) with per-query segments.

    subsets: optional list of per-query user-id arrays (rkr_query_exact_subsets).
    member: optional (nq, (n + 31) // 32) uint32 subset bitmaps (rkr_query_exact_bitmap)."""
    lib = load()
    nq, _ = _shape(Q)
    kk = np.broadcast_to(np.asarray(k if not _is_torch(k) else k.cpu().numpy(), np.int32), (nq,))
    off = np.concatenate([[0], np.cumsum(kk, dtype=np.int64)])
    pq, kq = _ptr(Q, np.float32)
    pk, kk_ = _ptr(k if _is_torch(k) else np.ascontiguousarray(kk), np.int32)
    users = _empty((int(off[-1]),), np.int32, device)
    ranks = _empty((int(off[-1]),), np.int32, device)
    pu, _ = _ptr(users, np.int32)
    pr, _ = _ptr(ranks, np.int32)
    stats = QueryStats()
    if member is not None:
        pm, words, km = _bitmap_ptr(member)
        _check(lib.rkr_query_exact_bitmap(index, pq, nq, pk, pm, words, pu, pr,
                                          ctypes.byref(stats), _stream(stream)))
    elif subsets is None:
        _check(lib.rkr_query_exact(index, pq, nq, pk, pu, pr, ctypes.byref(stats),
                                   _stream(stream)))
    else:
        so, su = _subsets_csr(subsets, nq)
        _check(lib.rkr_query_exact_subsets(index, pq, nq, pk, so.ctypes.data, su.ctypes.data, pu,
                                           pr, ctypes.byref(stats), _stream(stream)))
    return users, ranks, off, stats


def rkr_query_approx(index, Q, k, c: float, *, subsets=None, single: bool = False,
                     member=None, device: bool = False, stream=None):
    """c-approximate reverse k-ranks (Section 4.3): dict of per-user and per-query outputs.

    subsets: optional list of per-query user-id arrays (rkr_query_approx_subsets).
    single: answer the queries one at a time (rkr_query_approx_single)."""
    lib = load()
    nq, _ = _shape(Q)
    kk = np.broadcast_to(np.asarray(k if not _is_torch(k) else k.cpu().numpy(), np.int32), (nq,))
    off = np.concatenate([[0], np.cumsum(kk, dtype=np.int64)])
    tot = int(off[-1])
    pq, kq = _ptr(Q, np.float32)
    pk, kk_ = _ptr(k if _is_torch(k) else np.ascontiguousarray(kk), np.int32)
    out = dict(users=_empty((tot,), np.int32, device), n_low=_empty((tot,), np.uint32, device),
               n_up=_empty((tot,), np.uint32, device), est=_empty((tot,), np.float64, device),
               case=_empty((nq,), np.int32, device), nc=_empty((nq,), np.int32, device))
    ptrs = [_ptr(out[name], dt)[0] for name, dt in
            (("users", np.int32), ("n_low", np.uint32), ("n_up", np.uint32),
             ("est", np.float64), ("case", np.int32), ("nc", np.int32))]
    stats = QueryStats()
    if member is not None:
        pm, words, km = _bitmap_ptr(member)
        _check(lib.rkr_query_approx_bitmap(index, pq, nq, pk, pm, words, ctypes.c_double(c),
                                           *ptrs, ctypes.byref(stats), _stream(stream)))
    elif single:
        if subsets is not None:
            raise ValueError("the one-at-a-time mode takes no subsets")
        _check(lib.rkr_query_approx_single(index, pq, nq, pk, ctypes.c_double(c), *ptrs,
                                           ctypes.byref(stats), _stream(stream)))
    elif subsets is None:
        _check(lib.rkr_query_approx(index, pq, nq, pk, ctypes.c_double(c), *ptrs,
                                    ctypes.byref(stats), _stream(stream)))
    else:
        so, su = _subsets_csr(subsets, nq)
        _check(lib.rkr_query_approx_subsets(index, pq, nq, pk, so.ctypes.data, su.ctypes.data,
                                            ctypes.c_double(c), *ptrs, ctypes.byref(stats),
                                            _stream(stream)))
    out["offsets"] = off
    out["stats"] = stats
    return out


def rkr_query_approx_single(index, Q, k, c: float, **kw):
    """rkr_query_approx answered one query at a time (latency mode)."""
    return rkr_query_approx(index, Q, k, c, single=True, **kw)


def rkr_query_approx_candidates(index, Q, k, *, user_offset: int = 0, capacity=None,
                                stream=None):
    """Per-query candidates of one part of a sharded user set (rkr_query_approx_candidates):
    dict of offsets (nq + 1) and per-candidate users (global ids), n_low, n_up, est."""
    lib = load()
    nq, _ = _shape(Q)
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    pq, kq = _ptr(Q, np.float32)
    cap = int(capacity) if capacity is not None else int(max(1024, 16 * kk.sum()))
    while True:
        offs = np.empty(nq + 1, np.int64)
        out = dict(users=np.empty(cap, np.int32), n_low=np.empty(cap, np.uint32),
                   n_up=np.empty(cap, np.uint32), est=np.empty(cap, np.float64))
        st = lib.rkr_query_approx_candidates(
            index, pq, nq, kk.ctypes.data, int(user_offset), cap, offs.ctypes.data,
            out["users"].ctypes.data, out["n_low"].ctypes.data, out["n_up"].ctypes.data,
            out["est"].ctypes.data, _stream(stream))
        if st == 2 and capacity is None and offs[-1] > cap:   # RKR_ENOMEM: grow and retry
            cap = int(offs[-1])
            continue
        _check(st)
        tot = int(offs[-1])
        res = {key: v[:tot] for key, v in out.items()}
        res["offsets"] = offs
        return res


def rkr_merge_approx(k, c: float, s: int, offs, users, n_low, n_up, est) -> dict:
    """Steps 1-3 of Section 4.3 on the union of the parts' candidates (host code)."""
    lib = load()
    offs = np.ascontiguousarray(offs, np.int64)
    nq = len(offs) - 1
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    ins = [np.ascontiguousarray(a, dt) for a, dt in ((users, np.int32), (n_low, np.uint32),
                                                     (n_up, np.uint32), (est, np.float64))]
    tot = int(kk.sum(dtype=np.int64))
    out = dict(users=np.empty(tot, np.int32), n_low=np.empty(tot, np.uint32),
               n_up=np.empty(tot, np.uint32), est=np.empty(tot, np.float64),
               case=np.empty(nq, np.int32), nc=np.empty(nq, np.int32))
    _check(lib.rkr_merge_approx(nq, kk.ctypes.data, ctypes.c_double(c), int(s), offs.ctypes.data,
                                *[a.ctypes.data for a in ins],
                                *[out[key].ctypes.data for key in
                                  ("users", "n_low", "n_up", "est", "case", "nc")]))
    out["offsets"] = np.concatenate([[0], np.cumsum(kk, dtype=np.int64)])
    return out


def rkr_merge_exact(k, offs, users, ranks):
    """Def. 2 on the union of the parts' answers (host code): (users, ranks, offsets)."""
    lib = load()
    offs = np.ascontiguousarray(offs, np.int64)
    nq = len(offs) - 1
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    u = np.ascontiguousarray(users, np.int32)
    r = np.ascontiguousarray(ranks, np.int32)
    tot = int(kk.sum(dtype=np.int64))
    ou, orr = np.empty(tot, np.int32), np.empty(tot, np.int32)
    _check(lib.rkr_merge_exact(nq, kk.ctypes.data, offs.ctypes.data, u.ctypes.data, r.ctypes.data,
                               ou.ctypes.data, orr.ctypes.data))
    return ou, orr, np.concatenate([[0], np.cumsum(kk, dtype=np.int64)])


def rkr_query_exact_subsets(index, Q, k, subsets, **kw):
    """rkr_query_exact restricted to one user subset per query."""
    return rkr_query_exact(index, Q, k, subsets=subsets, **kw)


def rkr_query_approx_subsets(index, Q, k, subsets, c: float, **kw):
    """rkr_query_approx restricted to one user subset per query."""
    return rkr_query_approx(index, Q, k, c, subsets=subsets, **kw)


def rkr_rank_pairs(index, Q, pair_user, pair_query, *, stream=None):
    """Exact ranks (Def. 1) of (user, query) pairs; queries are rows of Q."""
    lib = load()
    nq, _ = _shape(Q)
    pq, kq = _ptr(Q, np.float32)
    u = np.ascontiguousarray(pair_user, np.int32)
    q = np.ascontiguousarray(pair_query, np.int32)
    out = np.empty(len(u), np.int32)
    _check(lib.rkr_rank_pairs(index, pq, nq, len(u), u.ctypes.data, q.ctypes.data,
                              out.ctypes.data, _stream(stream)))
    return out


def rkr_pair_features(index, R, Q, pair_user, pair_query, *, stream=None):
    """The pruner's inputs for pairs: (X (npairs x 65), t (npairs))."""
    lib = load()
    nq, _ = _shape(Q)
    R = np.ascontiguousarray(R, np.float32)
    pq, kq = _ptr(Q, np.float32)
    u = np.ascontiguousarray(pair_user, np.int32)
    q = np.ascontiguousarray(pair_query, np.int32)
    X = np.empty((len(u), 65), np.float32)
    t = np.empty(len(u), np.float32)
    _check(lib.rkr_pair_features(index, R.ctypes.data, pq, nq, len(u), u.ctypes.data,
                                 q.ctypes.data, X.ctypes.data, t.ctypes.data, _stream(stream)))
    return X, t


def rkr_query_exact_learned(index, pruner, R, Q, k, keep, *, certify: bool = True,
                            stream=None):
    """Def. 2 with the candidates of query i cut to keep[i] (an int or one per query)
    by the pruner's predictions; certify=True adds the exact fallback."""
    lib = load()
    nq, _ = _shape(Q)
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    kp = np.ascontiguousarray(np.broadcast_to(np.asarray(keep, np.int32), (nq,)))
    off = np.concatenate([[0], np.cumsum(kk, dtype=np.int64)])
    R = np.ascontiguousarray(R, np.float32)
    pq, kq = _ptr(Q, np.float32)
    users = np.empty(int(off[-1]), np.int32)
    ranks = np.empty(int(off[-1]), np.int32)
    stats = QueryStats()
    _check(lib.rkr_query_exact_learned(index, pruner._h, R.ctypes.data, pq, nq, kk.ctypes.data,
                                       kp.ctypes.data, int(bool(certify)), users.ctypes.data,
                                       ranks.ctypes.data, ctypes.byref(stats), _stream(stream)))
    return users, ranks, off, stats


def rkr_screen_scores(U, X, *, split: bool = False, stream=None):
    """Tensor-core screened scores and their error bounds for every pair (n x mx each)."""
    lib = load()
    n, d = _shape(U)
    mx, dx = _shape(X)
    if dx != d:
        raise RKRError(1, f"X has {dx} columns, U has {d}")
    _same_device(U, X)
    pu, ku = _ptr(U, np.float32)
    px, kx = _ptr(X, np.float32)
    s = np.empty((n, mx), dtype=np.float32)
    b = np.empty((n, mx), dtype=np.float32)
    _check(lib.rkr_screen_scores(pu, n, px, mx, d, int(split), s.ctypes.data_as(ctypes.c_void_p),
                                 b.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return s, b


def rkr_screen_scores_static(U, X, out_s, out_b, *, split: bool = False, stream=None):
    """rkr_screen_scores into caller-owned device buffers, with no device allocation.

    U (n x d), X (mx x d), out_s and out_b (n x mx, float32) must be CUDA tensors."""
    lib = load()
    n, d = _shape(U)
    mx, dx = _shape(X)
    if dx != d:
        raise RKRError(1, f"X has {dx} columns, U has {d}")
    for t in (U, X, out_s, out_b):
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()
                and str(t.dtype) == "torch.float32"):  # noqa: E129
            raise RKRError(1, "rkr_screen_scores_static takes contiguous float32 CUDA tensors")
    import torch
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (U, X, out_s, out_b)):
        raise RKRError(1, f"every tensor must be on the current device cuda:{dev}")
    if tuple(out_s.shape) != (n, mx) or tuple(out_b.shape) != (n, mx):
        raise RKRError(1, "output shape must be (n, mx)")
    _check(lib.rkr_screen_scores_static(U.data_ptr(), n, X.data_ptr(), mx, d, int(split),
                                        out_s.data_ptr(), out_b.data_ptr(), _stream(stream)))


class Pruner:
    """The learned pruner's monotone rank regressor (rkr_pruner_*): F features, H hidden."""

    def __init__(self, F: int = 65, H: int = 256, seed: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.rkr_pruner_create(F, H, seed, ctypes.byref(h)))
        self._h, self.F, self.H = h, F, H
        self.nparams = int(lib.rkr_pruner_nparams(h))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparams, np.float32)
        _check(load().rkr_pruner_params(self._h, 0, a.ctypes.data, self.nparams))
        return a

    def set_params(self, a) -> None:
        a = np.ascontiguousarray(a, np.float32)
        _check(load().rkr_pruner_params(self._h, 1, a.ctypes.data, self.nparams))

    def forward(self, X, t) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        y = np.empty(len(t), np.float32)
        _check(load().rkr_pruner_forward(self._h, X.ctypes.data, t.ctypes.data, len(t),
                                         y.ctypes.data, None))
        return y

    def loss_grads(self, X, t, target):
        X = np.ascontiguousarray(X, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        target = np.ascontiguousarray(target, np.float32)
        g = np.empty(self.nparams, np.float32)
        loss = ctypes.c_float()
        _check(load().rkr_pruner_loss_grads(self._h, X.ctypes.data, t.ctypes.data,
                                            target.ctypes.data, len(t), ctypes.byref(loss),
                                            g.ctypes.data, None))
        return float(loss.value), g

    def train(self, X, t, target, *, epochs=2, batch=4096, lr=1e-3, seed=0) -> float:
        X = np.ascontiguousarray(X, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        target = np.ascontiguousarray(target, np.float32)
        loss = ctypes.c_float()
        _check(load().rkr_pruner_train(self._h, X.ctypes.data, t.ctypes.data, target.ctypes.data,
                                       len(t), epochs, batch, lr, seed, ctypes.byref(loss), None))
        return float(loss.value)

    def invert(self, index, R, G: int = 64, stream=None) -> None:
        """Tabulate the network per user of `index` (an Index) on G points of t
        (rkr_pruner_invert); learned queries on that index with the same R then
        predict by table lookup.  G = 0 drops the tables."""
        R = np.ascontiguousarray(R, np.float32)
        _check(load().rkr_pruner_invert(self._h, index._h, R.ctypes.data, int(G),
                                        _stream(stream)))

    def table(self, n: int, G: int):
        """The tables of invert: (tab (n x G), grid (n x 2): t_0 and step per user)."""
        tab = np.empty((n, G), np.float32)
        grid = np.empty((n, 2), np.float32)
        _check(load().rkr_pruner_table(self._h, n, G, tab.ctypes.data, grid.ctypes.data))
        return tab, grid

    def save(self, path: str) -> None:
        """Write F, H and the weights to a file (rkr_pruner_save)."""
        _check(load().rkr_pruner_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Pruner":
        """A pruner read from a file written by save (rkr_pruner_load)."""
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.rkr_pruner_load(os.fsencode(path), ctypes.byref(h)))
        obj = cls.__new__(cls)
        obj._h = h
        obj.nparams = int(lib.rkr_pruner_nparams(h))
        a = np.empty(obj.nparams, np.float32)
        _check(lib.rkr_pruner_params(h, 0, a.ctypes.data, obj.nparams))
        obj.F, obj.H = None, None
        return obj

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().rkr_pruner_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Session:
    """One query per call with a captured CUDA graph (rkr_session_*)."""

    def __init__(self, index: "Index", max_k: int, c: float = 2.0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.rkr_session_create(index._h, int(max_k), ctypes.c_double(c), None,
                                      ctypes.byref(h)))
        self._h, self.max_k, self.index = h, int(max_k), index

    def query(self, q, k: int) -> dict:
        """Answer one query (a d-vector, numpy or CUDA tensor); outputs as numpy arrays."""
        pq, kq = _ptr(q, np.float32)
        out = dict(users=np.empty(k, np.int32), n_low=np.empty(k, np.uint32),
                   n_up=np.empty(k, np.uint32), est=np.empty(k, np.float64),
                   case=np.empty(1, np.int32), nc=np.empty(1, np.int32))
        _check(load().rkr_session_query(self._h, pq, int(k),
                                        *[out[key].ctypes.data for key in
                                          ("users", "n_low", "n_up", "est", "case", "nc")]))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().rkr_session_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


@dataclass
class _Info:
    n: int
    m: int
    d: int
    tau: int
    omega: int
    s: int
    nsamp: int
    xg: int


class Index:
    """Owns one index handle; see rkr_build for the parameters."""

    def __init__(self, U, P, **kw):
        self._h: Optional[ctypes.c_void_p] = rkr_build(U, P, **kw)
        self._read_info()

    def _read_info(self):
        raw = (ctypes.c_int64 * 8)()
        _check(load().rkr_index_info(self._h, raw))
        self.info = _Info(*[int(v) for v in raw])

    def device_bytes(self) -> int:
        """Device memory the index holds (rkr_index_device_bytes)."""
        out = ctypes.c_int64()
        _check(load().rkr_index_device_bytes(self._h, ctypes.byref(out)))
        return int(out.value)

    def save(self, path: str) -> None:
        """Write the index to a file (rkr_index_save)."""
        _check(load().rkr_index_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Index":
        """An index read from a file written by save (rkr_index_load)."""
        h = ctypes.c_void_p()
        _check(load().rkr_index_load(os.fsencode(path), ctypes.byref(h)))
        obj = cls.__new__(cls)
        obj._h = h
        obj._read_info()
        return obj

    def query_exact(self, Q, k, **kw):
        return rkr_query_exact(self._h, Q, k, **kw)

    def query_approx(self, Q, k, c, **kw):
        return rkr_query_approx(self._h, Q, k, c, **kw)

    def rank_pairs(self, Q, pair_user, pair_query, **kw):
        return rkr_rank_pairs(self._h, Q, pair_user, pair_query, **kw)

    def pair_features(self, R, Q, pair_user, pair_query, **kw):
        return rkr_pair_features(self._h, R, Q, pair_user, pair_query, **kw)

    def autotune(self, Q, k, **kw):
        return rkr_autotune(self._h, Q, k, **kw)

    def query_approx_candidates(self, Q, k, **kw):
        return rkr_query_approx_candidates(self._h, Q, k, **kw)

    def query_exact_learned(self, pruner, R, Q, k, keep, **kw):
        return rkr_query_exact_learned(self._h, pruner, R, Q, k, keep, **kw)

    def export(self, what: str) -> np.ndarray:
        i = self.info
        shapes = dict(perm=((i.m,), np.int32), fmin=((i.n,), np.float64),
                      fmax=((i.n,), np.float64), table=((i.n, i.tau), np.uint32),
                      samples=((i.nsamp,), np.int32), xlo=((i.n, i.xg), np.uint32),
                      xhi=((i.n, i.xg), np.uint32),
                      xgrid=((i.n, 2), np.float64), pnorm=((i.m,), np.float64),
                      dlo=((i.n, DEEP_GRID), np.uint32), dhi=((i.n, DEEP_GRID), np.uint32),
                      dgrid=((i.n, 2), np.float64))
        shape, dt = shapes[what]
        a = np.empty(shape, dtype=dt)
        _check(load().rkr_index_export(self._h, EXPORTS[what], a.ctypes.data_as(ctypes.c_void_p),
                                       a.nbytes))
        return a

    def timings(self) -> dict:
        """Device time (ms) of the build stages."""
        raw = (ctypes.c_double * 8)()
        _check(load().rkr_index_timings(self._h, raw, 8))
        names = ("items", "samples", "fbounds", "table", "levels", "exact_table", "total")
        return {k: float(raw[i]) for i, k in enumerate(names)}

    def close(self):
        if self._h is not None:
            load().rkr_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

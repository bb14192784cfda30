"""Thin ctypes binding of libcombsieve.so (include/combsieve.h).

Argument marshalling only: every step of the sieve runs in the CUDA library.
The functions keep the C names; `Plan` wraps a cs_plan_t for convenience.
If the library is missing, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcombsieve.so")

CS_OK = 0
CS_EINVAL = -1
CS_ENOMEM = -2
CS_EDEVICE = -3
CS_ETIMEOUT = -4
CS_ESTATE = -5
CS_ESIZE = -6
CS_EOVERFLOW = -7
CS_EAGAIN = -8

_NAMES = {0: "CS_OK", -1: "CS_EINVAL", -2: "CS_ENOMEM", -3: "CS_EDEVICE", -4: "CS_ETIMEOUT",
          -5: "CS_ESTATE", -6: "CS_ESIZE", -7: "CS_EOVERFLOW", -8: "CS_EAGAIN"}

# every symbol include/combsieve.h declares
EXPORTS = ("cs_plan", "cs_sieve", "cs_sync", "cs_info", "cs_fetch_bitset", "cs_counts", "cs_stats",
           "cs_rows", "cs_columns", "cs_device_bitset", "cs_kernel_times", "cs_destroy",
           "cs_last_error", "cs_primes", "cs_k_mod_p", "cs_modsolve", "cs_primes_static",
           "cs_batch_create", "cs_batch_run", "cs_batch_sync", "cs_batch_info", "cs_batch_destroy",
           "cs_server_start", "cs_submit", "cs_poll", "cs_server_plan", "cs_release", "cs_server_usage",
           "cs_server_stop", "cs_fetch_rows", "cs_cache_create", "cs_cache_fill", "cs_cache_info",
           "cs_cache_destroy", "cs_plan_cached", "cs_autotune", "cs_row_columns", "cs_issue_rate",
           "cs_atomic_rate")


class CSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class cs_tuning(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_uint64), ("tile_rows", ctypes.c_uint32),
                ("large_mode", ctypes.c_uint32), ("no_wheel", ctypes.c_uint32),
                ("large_grid", ctypes.c_uint32), ("chunk_numbers", ctypes.c_uint64),
                ("profile", ctypes.c_uint32), ("layout", ctypes.c_uint32), ("m_classes", ctypes.c_uint32),
                ("item_hits", ctypes.c_uint32), ("class_min_hits", ctypes.c_uint32),
                ("class_item_hits", ctypes.c_uint32), ("hit_buckets", ctypes.c_uint32),
                ("band_rows_log", ctypes.c_uint32), ("bucket_records", ctypes.c_uint64),
                ("walk_prep", ctypes.c_uint32)]


class cs_info_t(ctypes.Structure):
    _fields_ = [("M_c", ctypes.c_uint64), ("W", ctypes.c_uint64), ("words_per_row", ctypes.c_uint64),
                ("bitset_bytes", ctypes.c_uint64), ("S", ctypes.c_uint64), ("threshold", ctypes.c_uint64),
                ("tile_rows", ctypes.c_uint32), ("large_mode", ctypes.c_uint32),
                ("narrow", ctypes.c_uint32), ("wheel", ctypes.c_uint32),
                ("n_large_chunks", ctypes.c_uint64), ("launches_per_sieve", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("est_cost", ctypes.c_uint64), ("layout", ctypes.c_uint32), ("n_classes", ctypes.c_uint32),
                ("m_mod", ctypes.c_uint32), ("m_walked", ctypes.c_uint32), ("split_chunks", ctypes.c_uint64),
                ("item_mod", ctypes.c_uint32), ("item_classes", ctypes.c_uint32),
                ("item_chunks", ctypes.c_uint64), ("hit_buckets", ctypes.c_uint32), ("n_bands", ctypes.c_uint32),
                ("bucket_bytes", ctypes.c_uint64), ("apply_launches", ctypes.c_uint64),
                ("prep_chunks", ctypes.c_uint64)]


class cs_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("F", "F_small", "F_large", "solves", "levels", "hits_all",
                                               "n_small_primes", "n_large_primes", "survivors", "hash",
                                               "bucket_records")]


_lock = threading.Lock()
_lib = None


def load(path: Optional[str] = None):
    """Loads the CUDA library (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_2012_03771_gb300.build.build() "
                              "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        u32, u64, i32, sz, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
        P64 = ctypes.POINTER(ctypes.c_uint64)
        lib.cs_plan.argtypes = [u32, u64, u64, u64, u32, u64, ctypes.POINTER(cs_tuning), ctypes.POINTER(vp)]
        lib.cs_sieve.argtypes = [vp, vp]
        lib.cs_sync.argtypes = [vp]
        lib.cs_info.argtypes = [vp, ctypes.POINTER(cs_info_t)]
        lib.cs_fetch_bitset.argtypes = [vp, vp, sz]
        lib.cs_fetch_rows.argtypes = [vp, u64, u64, vp, sz]
        lib.cs_counts.argtypes = [vp, vp, sz, P64, P64]
        lib.cs_stats.argtypes = [vp, ctypes.POINTER(cs_stats_t)]
        lib.cs_rows.argtypes = [vp, vp, sz]
        lib.cs_columns.argtypes = [vp, vp, sz]
        lib.cs_row_columns.argtypes = [vp, u64, vp, sz, P64]
        lib.cs_device_bitset.argtypes = [vp]
        lib.cs_device_bitset.restype = vp
        lib.cs_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), P64]
        lib.cs_destroy.argtypes = [vp]
        lib.cs_last_error.argtypes = []
        lib.cs_last_error.restype = ctypes.c_char_p
        lib.cs_primes.argtypes = [u64, u64, vp, u64, P64, vp]
        lib.cs_primes_static.argtypes = [u64, u64, vp, u64, P64, vp]
        lib.cs_k_mod_p.argtypes = [u32, u64, vp, u64, vp, vp]
        lib.cs_modsolve.argtypes = [vp, vp, vp, vp, vp, u64, i32, vp]
        lib.cs_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(vp)]
        lib.cs_batch_run.argtypes = [vp, vp]
        lib.cs_batch_sync.argtypes = [vp]
        lib.cs_batch_info.argtypes = [vp, P64, P64]
        lib.cs_batch_destroy.argtypes = [vp]
        lib.cs_server_start.argtypes = [u64, i32, ctypes.POINTER(cs_tuning), ctypes.POINTER(vp)]
        lib.cs_submit.argtypes = [vp, u32, u64, u64, u64, u32, u64, P64]
        lib.cs_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int)]
        lib.cs_server_plan.argtypes = [vp, u64, ctypes.POINTER(vp)]
        lib.cs_release.argtypes = [vp, u64]
        lib.cs_server_usage.argtypes = [vp, P64, P64, P64]
        lib.cs_server_stop.argtypes = [vp]
        lib.cs_cache_create.argtypes = [u32, u64, u64, ctypes.POINTER(vp)]
        lib.cs_autotune.argtypes = [u32, u64, u64, u64, u32, u64, ctypes.c_char_p, ctypes.POINTER(cs_tuning)]
        lib.cs_cache_fill.argtypes = [vp, vp]
        lib.cs_cache_info.argtypes = [vp, P64, P64, P64]
        lib.cs_cache_destroy.argtypes = [vp]
        lib.cs_plan_cached.argtypes = [u32, u64, u64, u64, u32, u64, ctypes.POINTER(cs_tuning), vp,
                                       ctypes.POINTER(vp)]
        lib.cs_issue_rate.argtypes = [i32, u32, vp, u64, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_float)]
        lib.cs_atomic_rate.argtypes = [vp, u64, u32, vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_float)]
        for n in EXPORTS:
            if n not in ("cs_device_bitset", "cs_last_error"):
                getattr(lib, n).restype = i32
        _lib = lib
        return lib


def _check(rc: int):
    if rc != CS_OK:
        raise CSError(rc, load().cs_last_error().decode())
    return rc


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def make_tuning(threshold=0, tile_rows=0, large_mode=0, no_wheel=False, large_grid=0,
                chunk_numbers=0, profile=False, layout=0, m_classes=0, item_hits=0,
                class_min_hits=0, class_item_hits=0, hit_buckets=0, band_rows_log=0,
                bucket_records=0, walk_prep=0) -> cs_tuning:
    t = cs_tuning()
    t.walk_prep = walk_prep
    t.hit_buckets, t.band_rows_log, t.bucket_records = hit_buckets, band_rows_log, bucket_records
    t.layout = layout
    t.m_classes, t.item_hits, t.class_min_hits = m_classes, item_hits, class_min_hits
    t.class_item_hits = class_item_hits
    t.threshold, t.tile_rows, t.large_mode = threshold, tile_rows, large_mode
    t.no_wheel, t.large_grid, t.chunk_numbers = int(no_wheel), large_grid, chunk_numbers
    t.profile = int(profile)
    return t


# ------------------------------------------------------------ C-named calls

def cs_plan(P, d, M_start, M_inc, SL, L, tune: Optional[cs_tuning] = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().cs_plan(P, d, M_start, M_inc, SL, L, ctypes.byref(tune) if tune else None,
                          ctypes.byref(h)))
    return h


def cs_plan_status(P, d, M_start, M_inc, SL, L, tune: Optional[cs_tuning] = None) -> int:
    """Return code of cs_plan (the plan, if any, is destroyed)."""
    h = ctypes.c_void_p()
    rc = load().cs_plan(P, d, M_start, M_inc, SL, L, ctypes.byref(tune) if tune else None,
                        ctypes.byref(h))
    if rc == CS_OK:
        load().cs_destroy(h)
    return rc


def cs_sieve(plan, stream=None):
    _check(load().cs_sieve(plan, _stream_handle(stream)))


def cs_sync(plan):
    _check(load().cs_sync(plan))


def cs_info(plan) -> cs_info_t:
    out = cs_info_t()
    _check(load().cs_info(plan, ctypes.byref(out)))
    return out


def cs_fetch_bitset(plan, out: np.ndarray):
    _check(load().cs_fetch_bitset(plan, _ptr(out), out.size))
    return out


def cs_fetch_rows(plan, row0: int, out: np.ndarray):
    """Rows row0 .. row0 + out.shape[0] - 1 into out ([n, words_per_row] uint64)."""
    _check(load().cs_fetch_rows(plan, row0, out.shape[0], _ptr(out), out.size))
    return out


def cs_counts(plan, per_row: Optional[np.ndarray] = None):
    F, h = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().cs_counts(plan, _ptr(per_row) if per_row is not None else None,
                            per_row.size if per_row is not None else 0, ctypes.byref(F), ctypes.byref(h)))
    return int(F.value), int(h.value)


def cs_stats(plan) -> cs_stats_t:
    out = cs_stats_t()
    _check(load().cs_stats(plan, ctypes.byref(out)))
    return out


def cs_rows(plan, n: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(load().cs_rows(plan, _ptr(out), out.size))
    return out[:n]


def cs_columns(plan, n: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.int64)
    _check(load().cs_columns(plan, _ptr(out), out.size))
    return out[:n]


def cs_device_bitset(plan) -> int:
    return load().cs_device_bitset(plan) or 0


def cs_kernel_times(plan):
    ms = (ctypes.c_double * 7)()
    n = (ctypes.c_uint64 * 7)()
    _check(load().cs_kernel_times(plan, ms, n))
    return list(ms), list(n)


def cs_destroy(plan):
    _check(load().cs_destroy(plan))


def cs_last_error() -> str:
    return load().cs_last_error().decode()


def cs_primes(lo, hi, out_ptr: int, cap: int, stream=None) -> int:
    c = ctypes.c_uint64()
    _check(load().cs_primes(lo, hi, ctypes.c_void_p(out_ptr), cap, ctypes.byref(c), _stream_handle(stream)))
    return int(c.value)


def cs_primes_static(lo, hi, out_ptr: int, cap: int, stream=None) -> int:
    """cs_primes without device allocation (shared static scratch; see combsieve.h)."""
    c = ctypes.c_uint64()
    _check(load().cs_primes_static(lo, hi, ctypes.c_void_p(out_ptr), cap, ctypes.byref(c),
                                   _stream_handle(stream)))
    return int(c.value)


def cs_k_mod_p(P, d, p_ptr: int, n: int, r_ptr: int, stream=None):
    _check(load().cs_k_mod_p(P, d, ctypes.c_void_p(p_ptr), n, ctypes.c_void_p(r_ptr), _stream_handle(stream)))


def cs_modsolve(p_ptr, K_ptr, L_ptr, R_ptr, m_ptr, n, narrow, stream=None):
    _check(load().cs_modsolve(*(ctypes.c_void_p(x) for x in (p_ptr, K_ptr, L_ptr, R_ptr, m_ptr)),
                              n, int(narrow), _stream_handle(stream)))


def cs_issue_rate(mix: int, iters: int, sink_ptr: int, sink_words: int, stream=None):
    """(thread-level operations, milliseconds) of one integer issue-rate launch."""
    ops, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().cs_issue_rate(mix, iters, ctypes.c_void_p(sink_ptr), sink_words, _stream_handle(stream),
                                ctypes.byref(ops), ctypes.byref(ms)))
    return float(ops.value), float(ms.value)


def cs_atomic_rate(region_ptr: int, n_words: int, ops_per_thread: int, stream=None):
    """(atomic bit clears, milliseconds) of one scattered-clear launch over region_ptr[0 .. n_words)."""
    n, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().cs_atomic_rate(ctypes.c_void_p(region_ptr), n_words, ops_per_thread, _stream_handle(stream),
                                 ctypes.byref(n), ctypes.byref(ms)))
    return float(n.value), float(ms.value)


def cs_autotune(P, d, M_start, M_inc, SL, L, cache_path: Optional[str] = None) -> dict:
    """Tuning chosen by the library's autotuner (see combsieve.h)."""
    t = cs_tuning()
    _check(load().cs_autotune(P, d, M_start, M_inc, SL, L, cache_path.encode() if cache_path else None,
                              ctypes.byref(t)))
    return {"threshold": int(t.threshold), "tile_rows": int(t.tile_rows), "large_mode": int(t.large_mode),
            "item_hits": int(t.item_hits)}


# ---------------------------------------------------------------- wrapper

class Cache:
    """Device-resident primes and K mod p for one K = P#/d (cs_cache_*)."""

    def __init__(self, P, d, L_max):
        self.h = ctypes.c_void_p()
        self.key = (P, d)
        _check(load().cs_cache_create(P, d, L_max, ctypes.byref(self.h)))

    def fill(self, stream=None):
        _check(load().cs_cache_fill(self.h, _stream_handle(stream)))
        return self

    def info(self, count=False):
        n, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().cs_cache_info(self.h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(c) if count else None))
        return int(n.value), int(b.value), (int(c.value) if count else None)

    def close(self):
        if self.h:
            load().cs_cache_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """One sieve instance: owns a cs_plan_t and its device memory.  With
    cache=Cache(P, d, ...) its large primes come from the residue cache."""

    def __init__(self, P, d, M_start, M_inc, SL, L, cache=None, **tuning):
        self.params = (P, d, M_start, M_inc, SL, L)
        self.tuning = make_tuning(**tuning) if tuning else None
        if cache is None:
            self.h = cs_plan(P, d, M_start, M_inc, SL, L, self.tuning)
        else:
            self.h = ctypes.c_void_p()
            _check(load().cs_plan_cached(P, d, M_start, M_inc, SL, L,
                                         ctypes.byref(self.tuning) if self.tuning else None, cache.h,
                                         ctypes.byref(self.h)))
        self.cache = cache
        self.info = cs_info(self.h)

    @property
    def M_c(self):
        return self.info.M_c

    @property
    def W(self):
        return self.info.W

    @property
    def wpr(self):
        return self.info.words_per_row

    def sieve(self, stream=None):
        cs_sieve(self.h, stream)
        return self

    def sync(self):
        cs_sync(self.h)
        return self

    def bitset(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.M_c, self.wpr), dtype=np.uint64)
        cs_fetch_bitset(self.h, out.reshape(-1))
        return out

    def fetch_rows(self, row0, n):
        out = np.zeros((n, self.wpr), dtype=np.uint64)
        return cs_fetch_rows(self.h, row0, out)

    def counts(self):
        per_row = np.zeros(max(self.M_c, 1), dtype=np.uint32)
        F, h = cs_counts(self.h, per_row)
        return per_row[:self.M_c], F, h

    def stats(self):
        s = cs_stats(self.h)
        return {n: int(getattr(s, n)) for n, _ in cs_stats_t._fields_}

    def rows(self):
        return cs_rows(self.h, self.M_c)

    def columns(self):
        return cs_columns(self.h, self.W)

    def row_columns(self, row):
        """x values of one row's bits (the compact layout's differ by row)."""
        out = np.zeros(max(int(self.W), 1), dtype=np.int64)
        n = ctypes.c_uint64()
        _check(load().cs_row_columns(self.h, row, _ptr(out), out.size, ctypes.byref(n)))
        return out[:n.value]

    def kernel_times(self):
        return cs_kernel_times(self.h)

    def close(self):
        if self.h:
            cs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- batch / server

class Batch:
    """A CUDA-graph batch over existing plans (cs_batch_*); plans must outlive it."""

    def __init__(self, plans, n_streams=0):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        self.h = ctypes.c_void_p()
        _check(load().cs_batch_create(arr, len(self.plans), n_streams, ctypes.byref(self.h)))
        ns, nl = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().cs_batch_info(self.h, ctypes.byref(ns), ctypes.byref(nl)))
        self.n_streams, self.launches = int(ns.value), int(nl.value)

    def run(self, stream=None):
        _check(load().cs_batch_run(self.h, _stream_handle(stream)))
        return self

    def sync(self):
        _check(load().cs_batch_sync(self.h))
        return self

    def close(self):
        if self.h:
            load().cs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BorrowedPlan(Plan):
    def __init__(self, h):
        self.h = h
        self.info = cs_info(h)

    def close(self):
        self.h = None


class Server:
    """Continuous-batching request server (cs_server_*)."""

    def __init__(self, budget_bytes, max_slots=8, **tuning):
        self.h = ctypes.c_void_p()
        t = make_tuning(**tuning) if tuning else None
        _check(load().cs_server_start(budget_bytes, max_slots, ctypes.byref(t) if t else None,
                                      ctypes.byref(self.h)))

    def submit(self, P, d, M_start, M_inc, SL, L):
        """Ticket, or None when the request is not admitted now (CS_EAGAIN)."""
        t = ctypes.c_uint64()
        rc = load().cs_submit(self.h, P, d, M_start, M_inc, SL, L, ctypes.byref(t))
        if rc == CS_EAGAIN:
            return None
        _check(rc)
        return int(t.value)

    def poll(self, ticket) -> bool:
        done = ctypes.c_int()
        _check(load().cs_poll(self.h, ticket, ctypes.byref(done)))
        return bool(done.value)

    def plan(self, ticket) -> Plan:
        h = ctypes.c_void_p()
        _check(load().cs_server_plan(self.h, ticket, ctypes.byref(h)))
        return _BorrowedPlan(h)

    def release(self, ticket):
        _check(load().cs_release(self.h, ticket))

    def usage(self):
        u, b, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().cs_server_usage(self.h, ctypes.byref(u), ctypes.byref(b), ctypes.byref(r)))
        return int(u.value), int(b.value), int(r.value)

    def close(self):
        if self.h:
            load().cs_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

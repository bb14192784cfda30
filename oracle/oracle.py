"""Combined Sieve oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU code for what the sieve computes:

* ``sieve``: the traditional sieve of Section 2.1 with the cached K mod p of
  Section 3.1, implemented in plain C (oracle.c) and called through ctypes.
* ``G``: the modular-equation solver of Section 3.3 (Eq. modsol, cases a-E),
  written as the paper's recursion in Python integers.
* ``brute_force_bits``: bignum trial division of every N + x by every sieving
  prime (no modular shortcut), for tiny parameter sets.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may use this module.  Nothing here is imported by the CUDA path.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

EINVAL = -1
ENOMEM = -2


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_oracle.so with gcc (host code only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        u32, u64, i64, sz, c_int = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                    ctypes.c_size_t, ctypes.c_int)
        P64 = ctypes.POINTER(ctypes.c_uint64)
        PI64 = ctypes.POINTER(ctypes.c_int64)
        lib.or_validate.argtypes = [u32, u64, u64, u64, u32, u64]
        lib.or_validate.restype = c_int
        lib.or_columns.argtypes = [u32, u64, u32, PI64]
        lib.or_columns.restype = i64
        lib.or_rows.argtypes = [u64, u64, u64, P64]
        lib.or_rows.restype = i64
        lib.or_k_mod_p.argtypes = [u32, u64, P64, sz, P64]
        lib.or_k_mod_p.restype = c_int
        lib.or_sieve.argtypes = [u32, u64, u32, u64, u64, c_int, P64, sz, P64, P64, P64, c_int]
        lib.or_sieve.restype = c_int
        lib.or_hash.argtypes = [P64, sz, sz, u64]
        lib.or_hash.restype = u64
        lib.or_row_counts.argtypes = [P64, sz, sz, ctypes.POINTER(ctypes.c_uint32)]
        lib.or_row_counts.restype = None
        lib.or_prime_stats.argtypes = [u64, u64, P64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), c_int]
        lib.or_prime_stats.restype = c_int
        lib.or_primes.argtypes = [u64, u64, P64, sz]
        lib.or_primes.restype = i64
        _lib = lib
        return lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


class OracleError(ValueError):
    pass


# --------------------------------------------------------------- structure

def validate(P, d, M_start, M_inc, SL, L) -> int:
    """0 if the parameter set is accepted, EINVAL otherwise."""
    return _load().or_validate(P, d, M_start, M_inc, SL, L)


def columns(P: int, d: int, SL: int) -> np.ndarray:
    """Stored offsets x in [-SL, SL] with gcd(|x|, K) = 1, ascending (int64)."""
    out = np.zeros(2 * SL + 1, dtype=np.int64)
    W = _load().or_columns(P, d, SL, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if W < 0:
        raise OracleError(f"or_columns: {W}")
    return out[:W].copy()


def rows(d: int, M_start: int, M_inc: int) -> np.ndarray:
    """Multipliers m in [M_start, M_start + M_inc) with gcd(m, d) = 1 (uint64)."""
    out = np.zeros(max(M_inc, 1), dtype=np.uint64)
    n = _load().or_rows(d, M_start, M_inc, _p64(out))
    if n < 0:
        raise OracleError(f"or_rows: {n}")
    return out[:n].copy()


def k_mod_p(P: int, d: int, primes: Sequence[int]) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    r = np.zeros_like(p)
    rc = _load().or_k_mod_p(P, d, _p64(p), p.size, _p64(r))
    if rc:
        raise OracleError(f"or_k_mod_p: {rc}")
    return r


def sieve(P: int, d: int, SL: int, L: int, rows_m: Sequence[int], *, p_lo: Optional[int] = None,
          wheel: bool = True, threads: int = 0) -> Tuple[np.ndarray, np.ndarray, int]:
    """Traditional sieve of the given rows with primes max(P, p_lo) < p <= L.

    Returns (bits[n_rows, wpr] uint64, F_rows[n_rows] uint64, n_hit_primes)."""
    lib = _load()
    m = np.ascontiguousarray(np.asarray(rows_m, dtype=np.uint64))
    W = lib.or_columns(P, d, SL, None)
    if W < 0:
        raise OracleError(f"or_columns: {W}")
    wpr = (W + 63) // 64
    bits = np.zeros((max(m.size, 1), max(wpr, 1)), dtype=np.uint64)
    F = np.zeros(max(m.size, 1), dtype=np.uint64)
    nhit = ctypes.c_uint64(0)
    rc = lib.or_sieve(P, d, SL, P if p_lo is None else p_lo, L, 1 if wheel else 0, _p64(m), m.size,
                      _p64(bits), _p64(F), ctypes.byref(nhit), threads)
    if rc:
        raise OracleError(f"or_sieve: {rc}")
    return bits[:m.size, :wpr].copy(), F[:m.size].copy(), int(nhit.value)


def bitset_hash(bits: np.ndarray, row0: int = 0) -> int:
    """Position-dependent checksum of a [rows, wpr] uint64 bitset (see oracle.c)."""
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    n, wpr = b.shape if b.ndim == 2 else (0, 0)
    if n == 0 or wpr == 0:
        return 0
    return int(_load().or_hash(_p64(b), n, wpr, row0))


def row_counts(bits: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    n, wpr = b.shape
    out = np.zeros(n, dtype=np.uint32)
    if n and wpr:
        _load().or_row_counts(_p64(b), n, wpr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def prime_stats(lo: int, hi: int, threads: int = 0) -> Tuple[int, float, float]:
    """(number of primes in (lo, hi], sum log(1 - 1/p), sum 1/p)."""
    c = ctypes.c_uint64(0)
    lp = ctypes.c_double(0)
    inv = ctypes.c_double(0)
    rc = _load().or_prime_stats(lo, hi, ctypes.byref(c), ctypes.byref(lp), ctypes.byref(inv), threads)
    if rc:
        raise OracleError(f"or_prime_stats: {rc}")
    return int(c.value), float(lp.value), float(inv.value)


def primes(lo: int, hi: int) -> np.ndarray:
    """Primes in (lo, hi], ascending."""
    cap = max(16, int(1.3 * hi / max(math.log(max(hi, 3)), 1.0)) + 64)
    out = np.zeros(cap, dtype=np.uint64)
    n = _load().or_primes(lo, hi, _p64(out), cap)
    if n < 0:
        raise OracleError(f"or_primes: {n}")
    return out[:n].copy()


def compact_layout(P: int, d: int, SL: int, rows_m, bits: np.ndarray):
    """The compact layout written out from the literal one: row m keeps, in
    order, the literal columns x with gcd(m*K + x, d) = 1 (the offsets the wheel
    of d's primes would clear are not stored).  All rows are padded to
    ceil(W_max / 64) words, W_max the largest such column count over the
    residues rho of m mod d that are coprime to d.
    Returns (bits_compact, W_max, per-row column lists)."""
    xs = columns(P, d, SL)
    qd = [q for q in _simple_primes(P) if d % q == 0]
    K = 1
    for q in _simple_primes(P):
        if d % q:
            K *= q
    kq = {q: K % q for q in qd}

    def keep_mask(rho):
        keep = np.ones(xs.size, dtype=bool)
        for q in qd:
            keep &= ((rho * kq[q] + xs) % q) != 0
        return keep

    residues = [rho for rho in range(d) if math.gcd(rho, d) == 1]
    masks = {rho: keep_mask(rho) for rho in residues}
    W_max = max(int(m.sum()) for m in masks.values())
    wpr = (W_max + 63) // 64
    out = np.zeros((len(rows_m), max(wpr, 1)), dtype=np.uint64)
    cols = []
    for i, m in enumerate(rows_m):
        keep = masks[int(m) % d]
        lit = unpack_row(bits[i], xs.size)
        sel = lit[keep]
        packed = np.packbits(np.concatenate([sel, np.zeros(64 * wpr - sel.size, dtype=np.uint8)]).astype(np.uint8),
                             bitorder="little")
        out[i, :wpr] = packed.view("<u8")
        cols.append(xs[keep])
    return out[:, :wpr], W_max, cols


def full_sieve(P, d, M_start, M_inc, SL, L, *, wheel=True, threads=0):
    """Whole bitset of a parameter set: (m_of_row, bits, F_rows)."""
    if validate(P, d, M_start, M_inc, SL, L):
        raise OracleError("invalid parameter set")
    m = rows(d, M_start, M_inc)
    bits, F, _ = sieve(P, d, SL, L, m, wheel=wheel, threads=threads)
    return m, bits, F


# ------------------------------------------------ Section 3.3: G(p, K, L, R)

def G(p: int, K: int, L: int, R: int) -> int:
    """Smallest m >= 0 with L <= m*K mod p <= R (Eq. modfunc), by the case
    analysis of Eq. modsol.  Requires 0 <= L <= R < p and gcd(K, p) = 1.

    The nested term of case E is read as ceil((L + p * G(K, -p mod K, L mod K,
    R mod K)) / K): the parentheses printed in the equation are unbalanced and
    the derivation that follows it gives this form."""
    if K == 0 or L == 0:                                   # case a
        return 0
    if K >= p:                                             # case B
        return G(p, K % p, L, R)
    c = -(-L // K)
    if c <= R // K:                                        # case C
        return c
    if 2 * K >= p:                                         # case D
        return G(p, p - K, p - R, p - L)
    i = G(K, (-p) % K, L % K, R % K)                       # case E
    return -(-(L + p * i) // K)


def G_brute(p: int, K: int, L: int, R: int) -> int:
    """Smallest m >= 0 with L <= m*K mod p <= R, by trying m = 0, 1, 2, ..."""
    for m in range(p):
        if L <= (m * K) % p <= R:
            return m
    raise OracleError("no solution")


def large_prime_walk(p: int, r: int, M_start: int, M_inc: int, SL: int):
    """Hits of one large prime p > 2*SL over m in [M_start, M_start + M_inc),
    enumerated as in Section 3.2: from the current m, the next m whose interval
    p divides is found by one solve of Eq. modeq, i.e. G(p, r, p - v, p - v + 2*SL)
    where v = (m*r + SL) mod p.  Returns (list of (m, x), number of G calls)."""
    hits, solves = [], 0
    m, M_end = M_start, M_start + M_inc
    while m < M_end:
        v = (m * r + SL) % p
        if v <= 2 * SL:
            hits.append((m, SL - v))
            m += 1
            continue
        solves += 1
        m += G(p, r, p - v, p - v + 2 * SL)
    return hits, solves


# ------------------------------------------------- brute force (tiny cases)

def _simple_primes(n: int):
    if n < 2:
        return []
    comp = bytearray(n + 1)
    out = []
    for i in range(2, n + 1):
        if not comp[i]:
            out.append(i)
            for j in range(i * i, n + 1, i):
                comp[j] = 1
    return out


def brute_force_bits(P, d, M_start, M_inc, SL, L, wheel=True):
    """Every stored (m, x), trial-divided by every sieving prime with Python
    integers; no residues are cached.  Returns (m list, x list, bits as a
    list of lists of 0/1, F)."""
    small = _simple_primes(P)
    K = 1
    for q in small:
        if d % q:
            K *= q
    qd = [q for q in small if d % q == 0]
    ms = [m for m in range(M_start, M_start + M_inc) if math.gcd(m, d) == 1]
    xs = [x for x in range(-SL, SL + 1) if (math.gcd(abs(x), K) == 1 if x else K == 1)]
    sp = [p for p in _simple_primes(L) if p > P]
    grid, F = [], 0
    for m in ms:
        row = []
        for x in xs:
            n = m * K + x
            alive = 1
            for p in sp:
                if n % p == 0 and n != p:
                    alive = 0
                    F += 1
            if wheel:
                for q in qd:
                    if n % q == 0 and n != q:
                        alive = 0
            row.append(alive)
        grid.append(row)
    return ms, xs, grid, F


def pack_rows(grid, W):
    """0/1 lists -> [rows, ceil(W/64)] uint64 with column j at bit j & 63 of word j >> 6."""
    wpr = (W + 63) // 64
    out = np.zeros((len(grid), wpr), dtype=np.uint64)
    for i, row in enumerate(grid):
        for j, b in enumerate(row):
            if b:
                out[i, j >> 6] |= np.uint64(1 << (j & 63))
    return out


def unpack_row(words: np.ndarray, W: int) -> np.ndarray:
    bits = np.unpackbits(np.ascontiguousarray(words, dtype='<u8').view(np.uint8), bitorder="little")
    return bits[:W]

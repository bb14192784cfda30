"""Seeded synthetic workloads for the Combined Sieve.

This module only describes inputs: parameter tuples (P, d, M_start, M_inc, SL, L)
and seeded draws of them.  It holds none of the method's arithmetic, so both the
CUDA path and the CPU oracle may import it.

Parameter names follow the paper (Section 3 and the Runtime section):
  P        primorial bound; K = P#/d
  d        small squarefree divisor of P# (e.g. 210 = 7#)
  M_start  first multiplier m
  M_inc    number of consecutive m considered; only m with gcd(m, d) = 1 are rows
  SL       sieve half-length X; offsets x run over [-SL, SL] (interval S = 2*SL+1)
  L        sieve limit P_limit; sieving primes are P < p <= L
"""
from __future__ import annotations

import dataclasses
import random
from typing import Iterator, List


@dataclasses.dataclass(frozen=True)
class SieveParams:
    P: int
    d: int
    M_start: int
    M_inc: int
    SL: int
    L: int

    def as_tuple(self):
        return (self.P, self.d, self.M_start, self.M_inc, self.SL, self.L)

    def with_(self, **kw) -> "SieveParams":
        return dataclasses.replace(self, **kw)


# Small plain search: K = 503#/210, m in [1, 1001), X = 7000, primes up to 1e7.
PLAIN_503 = SieveParams(P=503, d=210, M_start=1, M_inc=1000, SL=7000, L=10**7)

# Paper-shaped single search around the 35,308 record gap (Section 1.1):
# K = 953#/210, m in [1e8, 1e8 + 1e5), X = 20000, primes up to 1e9.
SEARCH_953 = SieveParams(P=953, d=210, M_start=100_000_000, M_inc=100_000,
                         SL=20_000, L=10**9)

# Large single search around the 36,702 record gap (Section 1.1):
# K = 1019#/210, m in [1.64e8, 1.74e8), X = 25000, primes up to 1e11.
LARGE_1019 = SieveParams(P=1019, d=210, M_start=164_000_000, M_inc=10_000_000,
                         SL=25_000, L=10**11)

# The large search on a tenth of its m-range: the same 4.1e9 primes and the
# same chunks, a 477 MB bitset (still larger than L2); a shape small enough for
# hardware-counter captures of every launch.
LARGE_1019_M1E6 = LARGE_1019.with_(M_inc=1_000_000)

NAMED = {
    "plain_503": PLAIN_503,
    "search_953": SEARCH_953,
    "large_1019": LARGE_1019,
    "large_1019_m1e6": LARGE_1019_M1E6,
}

# Multipliers printed in Section 1.1 for the two record gaps.
RECORD_953 = (100_054_841, -9670, 35_308)      # m, offset of the gap's lower prime, gap
RECORD_1019 = (164_065_661, -18566, 36_702)

BATCH_SEED = 2012_03771


def batched_instances(n: int = 64, seed: int = BATCH_SEED) -> List[SieveParams]:
    """Independent searches of very uneven size: P uniform over {503, 701, 953, 1019},
    d uniform over {210, 2310}, M_inc log-uniform in [1e3, 1e6], SL uniform in
    [5000, 25000], L log-uniform in [1e8, 1e10], M_start log-uniform in [1e6, 1e8]."""
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        P = rng.choice((503, 701, 953, 1019))
        d = rng.choice((210, 2310))
        M_inc = int(10 ** rng.uniform(3, 6))
        SL = rng.randint(5000, 25000)
        L = int(10 ** rng.uniform(8, 10))
        M_start = int(10 ** rng.uniform(6, 8))
        out.append(SieveParams(P, d, M_start, M_inc, SL, L))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = BATCH_SEED + 1) -> List[float]:
    """Arrival times (seconds from 0) of a seeded Poisson stream."""
    rng = random.Random(seed)
    t, out = 0.0, []
    for _ in range(n):
        t += rng.expovariate(rate_per_s)
        out.append(t)
    return out


def tiny_cases(n: int, seed: int = 7) -> Iterator[SieveParams]:
    """Tiny parameter sets for brute-force checks: small primorials, small d,
    a few dozen m, narrow intervals, low sieve limits.  M_start = 1 gives
    N + x small enough that N + x can itself be a sieving prime; such draws may
    also violate the precondition M_start*K - SL >= 2, which the callers use to
    check that both implementations reject the same parameter sets."""
    rng = random.Random(seed)
    for _ in range(n):
        P = rng.choice((1, 2, 3, 5, 7, 13, 23, 37))
        ds = [1] + [c for c in (2, 6, 30, 210) if _primes_of(c)[-1] <= P]
        d = rng.choice(ds)
        SL = rng.randint(0, 120)
        M_start = 1 if rng.random() < 0.3 else SL + 2 + rng.randint(0, 40)
        M_inc = rng.randint(0, 30)
        L = rng.choice((0, 1, P, P + 1, 50, 500, 3000))
        yield SieveParams(P, d, M_start, M_inc, SL, L)


def _primes_of(c: int) -> List[int]:
    return [q for q in (2, 3, 5, 7) if c % q == 0] or [1]

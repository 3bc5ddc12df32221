"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds random draws only and none of the method's arithmetic:

* ``prime_draws``: raw integers in [2^30, 2^31); each side turns them into
  primes with its own primality test (next prime >= draw, repeats dropped).
* ``serving_requests``: the request stream of the serving workload (Poisson
  arrivals; lattice, width, height and prime count per request).

The method's only input besides these is (lattice, L, N, D), which needs no
generator: the state vector always starts at the all-singleton state.
"""
import numpy as np

PRIME_LO = 1 << 30
PRIME_HI = 1 << 31


def prime_draws(seed=0, count=64):
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.integers(PRIME_LO, PRIME_HI, size=count, dtype=np.int64)]


def serving_requests(seed=1, rate_per_s=200.0, n=10000, L_range=(4, 16), primes_range=(4, 16)):
    """List of dicts: arrival_s, lattice ('square'/'triangular'), L, N, n_primes,
    prime_seed.  L uniform in L_range, N uniform in {L, L+1}, n_primes uniform in
    primes_range (inclusive); each request draws its primes from its own seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    t = np.cumsum(gaps)
    lat = rng.integers(0, 2, size=n)
    L = rng.integers(L_range[0], L_range[1] + 1, size=n)
    dn = rng.integers(0, 2, size=n)
    npr = rng.integers(primes_range[0], primes_range[1] + 1, size=n)
    pseed = rng.integers(0, 2**31, size=n)
    return [dict(arrival_s=float(t[k]), lattice="square" if lat[k] == 0 else "triangular",
                 L=int(L[k]), N=int(L[k] + dn[k]), n_primes=int(npr[k]), prime_seed=int(pseed[k]))
            for k in range(n)]

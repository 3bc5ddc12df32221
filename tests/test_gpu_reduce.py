"""The gather kernels' exact modular reduction (Sec. 3.5: arithmetic modulo
primes below 2^31), driven on the GPU through cp_debug_reduce and compared
word by word with Python's %.  A destination word accumulates
v = sum_e coef_e x_e with x_e < p and sum_e |coef_e| < 2^20 (the table build's
bound), so the cases are the edges of |v| < p 2^20: +-(p S - 1) with
S = 2^20 - 1, multiples of p and their neighbours, and the largest primes."""
import random

import pytest

import paper_1005_3609_gb300 as cp
from paper_1005_3609_gb300 import _lib

import gpu_util

pytestmark = pytest.mark.gpu

S_MAX = (1 << 20) - 1


def _is_prime(n):
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def _largest_primes(count):
    out, p = [], (1 << 31) - 1
    while len(out) < count:
        if _is_prime(p):
            out.append(p)
        p -= 2
    return out


def _cases(p, rng):
    vals = [0, 1, -1, p * S_MAX - 1, -(p * S_MAX - 1), p - 1, 1 - p]
    for k in list(range(-64, 65)) + [S_MAX - 1, -(S_MAX - 1), S_MAX // 2, -(S_MAX // 2)]:
        vals += [k * p, k * p + 1, k * p - 1]
    vals += [rng.randrange(-(p * S_MAX - 1), p * S_MAX) for _ in range(4000)]
    return [v for v in vals if abs(v) < p << 20]


def test_reduction_matches_python_mod():
    rng = random.Random(5)
    primes = _largest_primes(8) + gpu_util.seed_primes(16) + [2, 3, 5, 65521, (1 << 30) + 3]
    values, mods = [], []
    for p in primes:
        for v in _cases(p, rng):
            values.append(v)
            mods.append(p)
    got = _lib.debug_reduce(values, mods)
    want = [v % p for v, p in zip(values, mods)]
    bad = [(v, p, g, w) for v, p, g, w in zip(values, mods, got, want) if g != w]
    assert not bad, bad[:5]


def test_reduction_rejects_out_of_range():
    p = (1 << 31) - 1
    with pytest.raises(cp.CPError):
        _lib.debug_reduce([p << 20], [p])
    with pytest.raises(cp.CPError):
        _lib.debug_reduce([0], [1 << 31])


def _halves_cases(p, rng):
    """(lo, hi) pairs of u = hi 2^16 + lo over (0, p 2^16), each u also split with lo
    near the ends of the 32-bit range (the sums' halves are not canonical)."""
    us = [1, 2, p - 1, p, p + 1, p * 65536 - 1, p * 65535, p * 65535 + 1, p * 65535 - 1]
    for k in list(range(1, 40)) + [32767, 32768, 65534, 65535]:
        us += [k * p - 1, k * p, k * p + 1]
    us += [rng.randrange(1, p * 65536) for _ in range(3000)]
    out = []
    for u in us:
        if not 0 < u < p * 65536:
            continue
        lo0, hi0 = u & 0xFFFF, u >> 16
        for j in (0, -1, 1, -32768, 32767, rng.randrange(-32768, 32768)):
            lo, hi = lo0 + j * 65536, hi0 - j
            if -(1 << 31) <= lo < (1 << 31) and -(1 << 31) <= hi < (1 << 31):
                out.append((lo, hi))
    return out


def test_halves_reduction_matches_python_mod():
    # the bulk-copy gather's 32-bit reduction (primes >= 2^17): full residues equal
    # Python's %, the stored signed representatives are congruent and in [-p, p)
    rng = random.Random(7)
    small = [p for p in range(1 << 17, (1 << 17) + 200) if _is_prime(p)][:3]
    primes = _largest_primes(8) + gpu_util.seed_primes(16) + small + [(1 << 30) + 3]
    assert all(_is_prime(p) for p in primes)
    lo, hi, mods = [], [], []
    for p in primes:
        for a, b in _halves_cases(p, rng):
            lo.append(a)
            hi.append(b)
            mods.append(p)
    us = [b * 65536 + a for a, b in zip(lo, hi)]
    got = _lib.debug_reduce_halves(lo, hi, mods, full=True)
    bad = [(u, p, g) for u, p, g in zip(us, mods, got) if g != u % p]
    assert not bad, bad[:5]
    got = _lib.debug_reduce_halves(lo, hi, mods, full=False)
    bad = [(u, p, g) for u, p, g in zip(us, mods, got) if not (-p <= g < p and (g - u) % p == 0)]
    assert not bad, bad[:5]


def test_halves_reduction_refuses_outside_its_domain():
    with pytest.raises(cp.CPError):
        _lib.debug_reduce_halves([1], [0], [65521])  # p below 2^17
    with pytest.raises(cp.CPError):
        _lib.debug_reduce_halves([0], [0], [(1 << 31) - 1])  # u = 0
    with pytest.raises(cp.CPError):
        _lib.debug_reduce_halves([0], [131101], [131101])  # u = p 2^16

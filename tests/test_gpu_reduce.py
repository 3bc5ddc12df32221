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

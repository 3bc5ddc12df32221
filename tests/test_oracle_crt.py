"""Pins of the oracle's prime selection and Chinese remaindering (Sec. 3.5)."""
import random

import synthetic_inputs
from oracle import crt


def test_small_primes():
    assert [n for n in range(60) if crt.is_prime(n)] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59]
    assert crt.is_prime(2147483647)          # 2^31 - 1
    assert not crt.is_prime(2147483649)      # 3 * 715827883
    assert crt.is_prime(1073741827)          # smallest prime above 2^30


def test_primes_from_draws():
    ps = crt.primes_from_draws(synthetic_inputs.prime_draws(0, 64), 16)
    assert len(set(ps)) == 16
    assert all((1 << 30) <= p < (1 << 31) and crt.is_prime(p) for p in ps)
    assert ps[:8] == crt.primes_from_draws(synthetic_inputs.prime_draws(0, 64), 8)


def test_crt_roundtrip_signed():
    rng = random.Random(7)
    ps = crt.primes_from_draws(synthetic_inputs.prime_draws(3, 64), 12)
    mod = 1
    for p in ps:
        mod *= p
    for _ in range(200):
        x = rng.randrange(-(mod // 2) + 1, mod // 2)
        rows = [[x % p] for p in ps]
        assert crt.crt_signed(rows, ps) == [x]

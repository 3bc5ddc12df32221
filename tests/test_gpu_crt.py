"""Exact integers through the library alone (Sec. 3.5): residues modulo several
primes, recombined by CRT on the GPU, with the two sufficiency checks --
Whitney's bound |c_j| <= C(|E|, j) against the prime product, and
stabilisation (the value must not change when the last prime is dropped).
Config 2 (square 12 x 13, full degree 155) and config 3 (triangular 13 x 14,
full degree 181) are compared with the oracle's exact integers
(tests/golden/, written from oracle/ only)."""
import math

import pytest

import golden_io
import gpu_util
import paper_1005_3609_gb300 as cp

pytestmark = pytest.mark.gpu


def edges(lattice, L, N):
    e = L * (N - 1) + N * (L - 1)
    return e + ((L - 1) * (N - 1) if lattice == "triangular" else 0)


def needed_primes(lattice, L, N, primes):
    """Fewest leading primes whose product covers 2 C(|E|, j) for every j."""
    bound = max(math.comb(edges(lattice, L, N), j) for j in range(L * N))
    prod = 1
    for k, p in enumerate(primes):
        prod *= p
        if prod > 2 * bound:
            return k + 1
    raise AssertionError("not enough primes")


@pytest.mark.parametrize("lattice,L,N", [("square", 12, 13), ("triangular", 13, 14)])
def test_read_integers_exact_or_refused(lattice, L, N):
    want = golden_io.ptilde(lattice, L, N)
    pool = gpu_util.seed_primes(20)
    k = needed_primes(lattice, L, N, pool)  # 10 for config 2, 16 for config 3
    with cp.Strip(lattice, L, pool[:k], max_degree=-1, max_rows=N) as s:
        s.advance(N - 1)
        assert s.read_integers() == want
    # the configured 8 primes are too few: the library says so instead of returning wrong integers
    with cp.Strip(lattice, L, pool[:8], max_degree=-1, max_rows=N) as s:
        s.advance(N - 1)
        with pytest.raises(cp.CPError) as ei:
            s.read_integers()
        assert ei.value.code == cp.CP_EPRIMES
        got, flags, rc = s.read_integers(strict=False)
        assert rc == cp.CP_EPRIMES
        prod = math.prod(pool[:8])
        for j, (g, c) in enumerate(zip(got, want)):
            assert (g - c) % prod == 0  # the residues are right: the integers are c_j modulo prod(primes)
            if abs(c) * 2 >= prod:
                assert flags[j] & 1, j  # a coefficient the product cannot hold is flagged by the bound


def test_read_integers_small_strip_and_truncation():
    primes = gpu_util.seed_primes(3)
    want = golden_io.ptilde("square", 5, 6)
    with cp.Strip("square", 5, primes, max_degree=-1, max_rows=6) as s:
        s.advance(5)
        assert s.read_integers() == want
    with cp.Strip("square", 5, primes, max_degree=10, max_rows=6) as s:
        s.advance(5)
        assert s.read_integers() == want[:11]


def test_crt_checked_flags():
    primes = gpu_util.seed_primes(4)
    prod3 = math.prod(primes[:3])
    vals = [0, 1, -1, 12345, prod3 // 2 - 1, -(prod3 // 2) + 1, prod3 // 2 + 7, -prod3]
    res = [[v % p for v in vals] for p in primes]
    ints, flags, rc = cp.crt_checked(res, primes)
    assert ints == vals
    assert rc == cp.CP_EPRIMES  # the last two need the fourth prime: not stable
    assert [f & 2 for f in flags] == [0, 0, 0, 0, 0, 0, 2, 2]
    # bound check: a bound beyond the product is flagged, one inside is not
    bits = [0] * 6 + [1] * 2
    _, flags, rc = cp.crt_checked([r[:6] for r in res], primes, bound_bits=bits[:6])
    assert rc == 0 and flags == [0] * 6
    prod_bits = math.prod(primes).bit_length()
    _, flags, rc = cp.crt_checked([r[:2] for r in res], primes, bound_bits=[prod_bits - 2, prod_bits - 1])
    assert flags == [0, 1] and rc == cp.CP_EPRIMES


def test_sweep_series_integers_checked():
    primes = gpu_util.seed_primes(4)
    import torch
    stream = torch.cuda.Stream()
    with cp.Sweep("square", 15, primes, stream, tile=4, prime_groups=1) as sw:
        sw.run()
        series = sw.series_integers()
        res = sw.read_series()
        assert series == [cp.crt(res[x], primes) for x in range(3)]
        t1 = golden_io.table1()
        assert series[0][: 2 * 15 - 4] == t1["alpha"][: 2 * 15 - 4]
    with cp.Sweep("square", 15, primes[:1], stream, tile=4, prime_groups=1) as sw:
        sw.run()
        with pytest.raises(cp.CPError) as ei:
            sw.series_integers()  # one prime can never be shown stable
        assert ei.value.code == cp.CP_EPRIMES

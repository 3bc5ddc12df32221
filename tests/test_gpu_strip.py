"""GPU parity of the strip path (cp_create_strip / cp_advance_rows / cp_read_coeffs) against the oracle.

Every comparison is bit-exact: residues per prime, and integers after CRT.
"""
import numpy as np
import pytest

import golden_io
import gpu_util
from oracle import modp, partitions, tm_exact

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()


def run_strip(lattice, L, N, primes, D=-1):
    with cp.Strip(lattice, L, primes, max_degree=D, max_rows=N) as s:
        s.advance(N - 1)
        return s.read()


# ---------------------------------------------------------------- state spaces

@pytest.mark.parametrize("m", range(1, 13))
def test_ncnnn_enumeration_matches_paper_order(m):
    got = [tuple(int(x) for x in row) for row in cp.debug_enumerate_space(0, m)]
    assert got == list(partitions.ncnnn_ordered(m))


def interleaved_order(m, e):
    """The library's order of the excepted space: NCNNN partitions in the paper's
    order, each one whose site e is alone (and e-1 !~ e+1) followed by its join
    with e+1.  Same set as the paper's ordering (Sec. 3.4), different bijection."""
    out = []
    for s in partitions.ncnnn_ordered(m):
        out.append(s)
        alone = all(s[i] != s[e] for i in range(m) if i != e)
        if alone and (e == 0 or s[e - 1] != s[e + 1]):
            out.append(tm_exact.join(s, e, e + 1)[0])
    return out


@pytest.mark.parametrize("m", range(2, 11))
def test_excepted_enumeration(m):
    for e in range(m - 1):
        got = [tuple(int(x) for x in row) for row in cp.debug_enumerate_space(1, m, e)]
        assert got == interleaved_order(m, e)
        assert sorted(got) == sorted(partitions.excepted_ordered(m, e))


@pytest.mark.parametrize("m", [13, 16, 18, 20])
def test_rank_unrank_bijection_large(m):
    bad, size = cp.debug_check_space(0, m)
    assert bad == 0 and size == partitions.motzkin(m - 1)
    for e in (0, m // 2, m - 2):
        bad, size = cp.debug_check_space(1, m, e)
        assert bad == 0 and size == partitions.motzkin(m - 1) + partitions.motzkin(m - 2)


# ---------------------------------------------------------------- rectangles

def test_config1_square_5x6_exact():
    primes = gpu_util.seed_primes(8)
    want = golden_io.ptilde("square", 5, 6)
    got = run_strip("square", 5, 6, primes)
    assert got.tolist() == gpu_util.residues_of(want, primes)
    assert cp.crt(got, primes) == want


@pytest.mark.parametrize("lattice,L,N,n_exact", [("square", 12, 13, 13), ("triangular", 13, 14, 19)])
def test_configs_2_3_full_polynomial(lattice, L, N, n_exact):
    want = golden_io.ptilde(lattice, L, N)
    primes8 = gpu_util.seed_primes(8)
    got = run_strip(lattice, L, N, primes8)
    assert got.tolist() == gpu_util.residues_of(want, primes8)
    # enough primes for the integers themselves (Whitney bound + stabilisation)
    primes = gpu_util.seed_primes(n_exact)
    got = run_strip(lattice, L, N, primes)
    assert cp.crt(got, primes) == want
    assert cp.crt(got[:-2], primes[:-2]) == want


def test_two_by_n_triangular_closed_form_all_heights():
    primes = gpu_util.seed_primes(4)
    with cp.Strip("triangular", 2, primes, max_degree=-1, max_rows=40) as s:
        for N in range(1, 41):
            if N > 1:
                s.advance(1)
            got = s.read()
            nv = 2 * N
            want = gpu_util.ptilde_of_q_product([[0, 1], [-1, 1]] + [[-2, 1]] * (2 * N - 2), nv)
            assert cp.crt(got[:, :nv], primes) == want, N
            assert not got[:, nv:].any()


def test_two_by_n_square_closed_form():
    primes = gpu_util.seed_primes(4)
    with cp.Strip("square", 2, primes, max_degree=-1, max_rows=30) as s:
        for N in range(1, 31):
            if N > 1:
                s.advance(1)
            want = gpu_util.ptilde_of_q_product([[0, 1], [-1, 1]] + [[3, -3, 1]] * (N - 1), 2 * N)
            assert cp.crt(s.read()[:, : 2 * N], primes) == want


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("L,N", [(1, 1), (1, 7), (7, 1), (2, 1), (3, 2), (4, 4), (6, 5), (8, 9), (9, 3)])
def test_small_rectangles_exact(lattice, L, N):
    primes = gpu_util.seed_primes(5)  # 5 primes: the 4-byte (unvectorised) path
    want = tm_exact.ptilde(lattice, L, N)
    got = run_strip(lattice, L, N, primes)
    assert got.tolist() == gpu_util.residues_of(want, primes)


@pytest.mark.parametrize("n_primes", [1, 2, 3, 4, 7, 8, 12, 16, 32])
def test_prime_counts(n_primes):
    primes = gpu_util.seed_primes(n_primes, seed=3)
    for lattice in ("square", "triangular"):
        want = tm_exact.ptilde(lattice, 6, 7)
        got = run_strip(lattice, 6, 7, primes)
        assert got.tolist() == gpu_util.residues_of(want, primes)


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_truncation_and_heights_against_modp_oracle(lattice):
    primes = gpu_util.seed_primes(8, seed=5)
    L, D, heights = 11, 20, [1, 2, 5, 11, 12, 16]
    ref = {p: modp.ptilde_heights(lattice, L, heights, D, p) for p in primes[:2]}
    with cp.Strip(lattice, L, primes, max_degree=D, max_rows=max(heights)) as s:
        h = 1
        for H in heights:
            s.advance(H - h)
            h = H
            assert s.height == H
            got = s.read()
            for k, p in enumerate(primes[:2]):
                assert got[k].tolist() == ref[p][H].tolist(), (H, p)


# the eight largest primes below 2^31: the modular reduction's correction step
# must not wrap around 2^32 when p is within a few thousand of 2^31
TOP_PRIMES = [2147483647, 2147483629, 2147483587, 2147483579, 2147483563, 2147483549, 2147483543, 2147483497]


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("n_primes", [8, 5])  # 16-byte rows (TMA gather) and 4-byte rows (register gather)
def test_primes_just_below_2_31(lattice, n_primes):
    primes = TOP_PRIMES[:n_primes]
    L, D, heights = 11, 30, [6, 12]
    with cp.Strip(lattice, L, primes, max_degree=D, max_rows=max(heights)) as s:
        h = 1
        for H in heights:
            s.advance(H - h)
            h = H
            got = s.read()
            for k, p in enumerate(primes):
                assert got[k].tolist() == modp.ptilde_heights(lattice, L, [H], D, p)[H].tolist(), (H, p)


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_transpose_symmetry(lattice):
    primes = gpu_util.seed_primes(4, seed=9)
    a = run_strip(lattice, 9, 12, primes, D=40)
    b = run_strip(lattice, 12, 9, primes, D=40)
    assert (a == b).all()


def test_degree_zero():
    primes = gpu_util.seed_primes(4)
    got = run_strip("square", 10, 10, primes, D=0)
    assert got.tolist() == [[1]] * 4


def test_invalid_arguments():
    primes = gpu_util.seed_primes(2)
    with pytest.raises(cp.CPError):
        cp.Strip("square", 0, primes)
    with pytest.raises(cp.CPError):
        cp.Strip("square", cp.CP_MAX_L + 1, primes)
    with pytest.raises(cp.CPError):
        cp.Strip("square", 4, [primes[0], primes[0]])
    with pytest.raises(cp.CPError):
        cp.Strip("square", 4, [(1 << 31) + 11])
    with cp.Strip("square", 3, primes, max_rows=3) as s:
        s.advance(2)
        with pytest.raises(cp.CPError):
            s.advance(1)


# ---------------------------------------------------------------- CRT and primes

def test_crt_roundtrip():
    rng = np.random.default_rng(1)
    primes = gpu_util.seed_primes(16)
    mod = 1
    for p in primes:
        mod *= p
    vals = [int(x) for x in rng.integers(-2**62, 2**62, size=50)]
    vals += [0, 1, -1, mod // 2, -(mod // 2) + 1, 12345678901234567890123456789 * 10**40]
    res = [[v % p for v in vals] for p in primes]
    assert cp.crt(res, primes) == vals


def test_select_primes_matches_oracle():
    import synthetic_inputs
    from oracle import crt as ocrt
    for seed in (0, 1, 7):
        draws = synthetic_inputs.prime_draws(seed, 128)
        assert cp.select_primes(draws, 24) == ocrt.primes_from_draws(draws, 24)


def test_wide_rows_eight_chunk_passes():
    # 32 primes x 136 coefficients: 1088 chunks of 16 bytes per row (the TMA kernel's 8-pass variant)
    primes = gpu_util.seed_primes(32, seed=21)
    want = tm_exact.ptilde("square", 8, 17)
    got = run_strip("square", 8, 17, primes)
    assert got.tolist() == gpu_util.residues_of(want, primes)


def test_strip_tiles_agree():
    # cp_strip_set_tile: the register kernel and TMA geometries give the same residues
    primes = gpu_util.seed_primes(16, seed=3)
    want = None
    for tile in (0, 4, 16 | (48 << 12) | (4 << 20) | (2 << 24), 64 | (64 << 12) | (8 << 20) | (1 << 24),
                 128 | (32 << 12) | (2 << 20) | (4 << 24)):
        with cp.Strip("square", 11, primes, max_degree=40, max_rows=8) as s:
            s.set_tile(tile)
            s.advance(7)
            got = s.read().tolist()
        if want is None:
            want = got
        assert got == want, tile
    with cp.Strip("square", 5, primes, max_degree=8, max_rows=2) as s:
        with pytest.raises(cp.CPError):
            s.set_tile(3)
        with pytest.raises(cp.CPError):
            s.set_tile(32 | (3 << 28))  # no block shape 3


@pytest.mark.parametrize("primes", [[3, 5, 7, 65521], [2, 131071, 2147483629, 2147483587],
                                    [131101, 131111, 2147483647, 1073741827]])
def test_small_and_large_primes_on_the_bulk_copy_kernel(primes):
    # four primes per 16-byte chunk (the TMA kernel); primes below 2^17 take the
    # 64-bit reduction of the word sums, all primes >= 2^17 the 32-bit one
    for lattice in ("square", "triangular"):
        want = gpu_util.residues_of(tm_exact.ptilde(lattice, 6, 6), primes)
        for tile in (0, 32 | (2 << 24), 16 | (8 << 20)):
            with cp.Strip(lattice, 6, primes, max_degree=-1, max_rows=6) as s:
                s.set_tile(tile)
                s.advance(5)
                assert s.read().tolist() == want, (lattice, hex(tile))


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_narrow_blocks_match_oracle(lattice):
    # 6 x 6 at full degree with 16 primes: rows of 36 degrees x 4 chunks = 144
    # chunks, which the default tile gathers with narrow blocks (5 consumer
    # warps); narrow blocks at every stage size and the forced wide block give
    # the oracle's residues
    primes = gpu_util.seed_primes(16, seed=11)
    want = gpu_util.residues_of(tm_exact.ptilde(lattice, 6, 6), primes)
    narrow, wide = 2 << 28, 1 << 28
    for tile in (0, 16 | (1 << 20) | narrow, 32 | (2 << 20) | (1 << 24) | narrow, 64 | (4 << 20) | narrow,
                 128 | (8 << 20) | (52 << 12) | narrow, 64 | (8 << 20) | (1 << 24) | wide, 32 | narrow | (2 << 24)):
        with cp.Strip(lattice, 6, primes, max_degree=-1, max_rows=6) as s:
            s.set_tile(tile)
            s.advance(5)
            assert s.read().tolist() == want, hex(tile)

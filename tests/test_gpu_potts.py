"""GPU tests of the any-v Potts strip (cp_create_strip_potts), Sec. 3.1-3.3.

The strip runs the plain transfer matrix T = (prod V_i)(prod H_{i,i+1}) on all
non-crossing partitions with integer v.  Its residues are compared bit for bit
with the oracle's any-v transfer matrix (``oracle.tm_generic``, itself pinned
to brute force over edge subsets), at v = -1 with the chromatic strip, and at
widths beyond the oracle with two identities that hold at any size:
Z(1, v) = (1 + v)^{|E|} (w = 1: every edge subset counts v^{|A|}) and
Z(q, 0) = q^{|V|} (Z~ = 1).
"""
import numpy as np
import pytest

import gpu_util
from oracle import partitions, tm_generic

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()


def run_potts(lattice, L, N, v, primes, D=-1):
    with cp.Strip(lattice, L, primes, max_degree=D, max_rows=N, v=v) as s:
        assert s.n_states == (partitions.catalan(L), partitions.catalan(L))
        s.advance(N - 1)
        return s.read()


def n_edges(lattice, L, N):
    e = L * (N - 1) + N * (L - 1)
    return e + (L - 1) * (N - 1) if lattice == "triangular" else e


# ---------------------------------------------------------------- state space

def catalan_order(lo, hi):
    """The library's order of the non-crossing partitions of points lo..hi-1, as
    block lists: the first point alone first, then by its smallest partner, the
    inner points the most significant digit, the right part the least."""
    if hi - lo <= 1:
        return [[[lo]]] if hi > lo else [[]]
    out = [[[lo]] + rest for rest in catalan_order(lo + 1, hi)]
    for j in range(lo + 1, hi):
        for inner in catalan_order(lo + 1, j):
            for right in catalan_order(j, hi):
                blk = [b for b in right if j in b][0]
                others = [b for b in right if j not in b]
                out.append([[lo] + blk] + inner + others)
    return out


@pytest.mark.parametrize("m", range(1, 10))
def test_catalan_enumeration(m):
    got = [tuple(int(x) for x in row) for row in cp.debug_enumerate_space(2, m)]
    want = [partitions.from_blocks(m, [[p for p in b] for b in blocks]) for blocks in catalan_order(0, m)]
    assert got == want
    every = sorted(s for s in partitions.all_partitions(m) if partitions.is_noncrossing(s))
    assert sorted(got) == every


@pytest.mark.parametrize("m", [12, 14, 16])
def test_catalan_bijection_large(m):
    bad, size = cp.debug_check_space(2, m)
    assert bad == 0 and size == partitions.catalan(m)


# ---------------------------------------------------------------- against the oracle

@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("v", [-2, 1, 2, 3])
def test_small_rectangles_match_oracle(lattice, v):
    primes = gpu_util.seed_primes(3, seed=7)
    for L in range(1, 7):
        for N in sorted({1, 2, L, L + 1}):
            want = tm_generic.ztilde(lattice, L, N, v)
            got = run_potts(lattice, L, N, v, primes)
            assert got.tolist() == gpu_util.residues_of(want, primes), (lattice, L, N, v)


@pytest.mark.parametrize("lattice,L,N,v,P", [
    ("square", 9, 4, 2, 8),        # 16-byte rows: the TMA gather, several tiles and a ragged tail
    ("square", 9, 4, -3, 5),       # odd prime count: the register gather
    ("triangular", 8, 4, -2, 4),
    ("triangular", 8, 3, 3, 7),
])
def test_wider_strips_match_oracle(lattice, L, N, v, P):
    primes = gpu_util.seed_primes(P, seed=11)
    want = tm_generic.ztilde(lattice, L, N, v)
    assert run_potts(lattice, L, N, v, primes).tolist() == gpu_util.residues_of(want, primes)


def test_truncated_degree():
    primes = gpu_util.seed_primes(4, seed=3)
    want = tm_generic.ztilde("square", 6, 6, 2)
    got = run_potts("square", 6, 6, 2, primes, D=9)
    assert got.tolist() == gpu_util.residues_of(want[:10], primes)


# ---------------------------------------------------------------- identities at any size

@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_v_minus_one_is_the_chromatic_strip(lattice):
    primes = gpu_util.seed_primes(8, seed=5)
    L, N = 11, 6
    chrom = None
    with cp.Strip(lattice, L, primes, max_rows=N) as s:
        s.advance(N - 1)
        chrom = s.read()
    assert np.array_equal(run_potts(lattice, L, N, -1, primes), chrom)


@pytest.mark.parametrize("lattice,L,N,v", [("square", 13, 3, 3), ("triangular", 12, 3, -2),
                                           ("square", 14, 2, 1)])
def test_w_equals_one_and_v_zero(lattice, L, N, v):
    primes = gpu_util.seed_primes(4, seed=9)
    got = run_potts(lattice, L, N, v, primes)
    for k, p in enumerate(primes):
        assert int(got[k].astype(np.int64).sum()) % p == pow(1 + v, n_edges(lattice, L, N), p)
    zero = run_potts(lattice, L, N, 0, primes)
    assert (zero[:, 0] == 1).all() and (zero[:, 1:] == 0).all()


def test_strip_reset_and_continue():
    primes = gpu_util.seed_primes(4, seed=2)
    with cp.Strip("triangular", 5, primes, max_rows=6, v=2) as s:
        s.advance(3)
        first = s.read()
        s.reset()
        s.advance(3)
        assert np.array_equal(s.read(), first)
        s.advance(2)
        assert s.read().tolist() == gpu_util.residues_of(tm_generic.ztilde("triangular", 5, 6, 2), primes)


# ---------------------------------------------------------------- errors

def test_rejections():
    primes = gpu_util.seed_primes(2)
    with pytest.raises(cp.CPError):
        cp.Strip("square", 4, primes, max_rows=2, v=17)  # |v| > CP_POTTS_MAX_V
    with pytest.raises(cp.CPError):
        cp.Strip("square", 17, primes, max_rows=2, v=1)  # L > CP_POTTS_MAX_L
    # 13 sites: 20 source bits, 10 coefficient bits; (1+v)^2 v = 4624 does not fit
    with pytest.raises(cp.CPError, match="does not fit"):
        cp.Strip("triangular", 13, primes, max_rows=2, v=16)
    # the library is still usable afterwards
    assert run_potts("square", 3, 3, 16, primes).tolist() == gpu_util.residues_of(
        tm_generic.ztilde("square", 3, 3, 16), primes)


def test_largest_coupling():
    # v = 16 at widths whose spaces leave 14 coefficient bits: (1+v)^2 v = 4624 fits
    primes = gpu_util.seed_primes(4, seed=12)
    for lattice, L, N in (("triangular", 8, 3), ("square", 9, 3)):
        want = tm_generic.ztilde(lattice, L, N, 16)
        assert run_potts(lattice, L, N, 16, primes).tolist() == gpu_util.residues_of(want, primes), lattice

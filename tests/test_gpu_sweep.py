"""GPU parity of the batched finite-lattice sweep (cp_sweep_*).

Small orders against the oracle (every rectangle's residues and every series
term, bit-exact); the full k = 33 sweeps against the values the paper prints
(Table 1, Baxter's product eq. (efb), eqs. (efs_ser)/(efc_ser)).
"""
import pytest

import golden_io
import gpu_util
from oracle import flm, graphs, modp, tm_exact

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")


@pytest.fixture(scope="module")
def stream():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()
    return torch.cuda.Stream()


def oracle_series(lattice, k, primes_for_crt=None):
    """Exact series from the oracle: flm_series on exact P~, plus the mu term (square, odd k)."""
    n = flm.n_terms(lattice, k) + (1 if lattice == "square" and k % 2 == 1 else 0)
    pt = {}
    for r in range(1, k // 2 + 1):
        hs = [s for rr, s in flm.band(k) if rr == r]
        got = tm_exact.ptilde_heights(lattice, r, hs, n - 1)
        pt.update({(r, s): got[s] for s in hs})
    b, s, c = flm.flm_series(lattice, k, pt, n)
    if lattice == "square" and k % 2 == 1:
        m = k // 2
        mu = flm.mu_series(2 * m)[2 * m]
        b[n - 1] += mu
        s[n - 1] -= m * mu
    return pt, (b, s, c)


@pytest.mark.parametrize("lattice,k,n_primes", [("square", 9, 3), ("square", 12, 4), ("triangular", 11, 5),
                                                ("square", 15, 8), ("triangular", 14, 8)])
def test_small_sweep_matches_oracle(stream, lattice, k, n_primes):
    primes = gpu_util.seed_primes(n_primes, seed=k)
    pt, series = oracle_series(lattice, k)
    with cp.Sweep(lattice, k, primes, stream, tile=4, prime_groups=1) as sw:
        assert sorted(sw.rects) == sorted(flm.band(k))
        sw.run()
        sw.sync()
        got = sw.read_ptilde()
        for rs, res in got.items():
            assert res.tolist() == gpu_util.residues_of(pt[rs][: sw.n_terms], primes), rs
        res = sw.read_series()
        for x in range(3):
            assert res[x].tolist() == gpu_util.residues_of(series[x], primes), x


@pytest.mark.parametrize("k", [16, 17])
def test_tile_and_group_choices_agree(stream, k):
    # k = 16: rows of 29 degrees (chunk counts that do not divide 256);
    # k = 17: rows of 32 degrees, so 16/8/4 primes give 128/64/32 chunks and the
    # TMA kernel runs 2, 4 and 8 consumer row groups
    primes = gpu_util.seed_primes(16, seed=2)
    ref = None
    # register kernel, TMA kernel with default stages, and every edges-per-stage x chunks-per-thread variant
    tma = [32 | (48 << 12) | (e << 20) | (c << 24) for e in (1, 2, 4, 8) for c in (1, 2, 4)]
    for tile in [1, 2, 4, 8, 16, 32, 64, 128] + tma:
        for groups in (1, 2, 4):
            with cp.Sweep("square", k, primes, stream, tile=tile, prime_groups=groups) as sw:
                sw.run()
                sw.sync()
                got = (sw.read_series().tobytes(), {k: v.tobytes() for k, v in sw.read_ptilde().items()})
            if ref is None:
                ref = got
            assert got == ref, (tile, groups)


def test_repeated_runs_identical(stream):
    primes = gpu_util.seed_primes(8, seed=4)
    with cp.Sweep("triangular", 12, primes, stream, tile=2, prime_groups=2) as sw:
        sw.run()
        a = sw.read_series()
        sw.run()
        sw.run()
        assert (sw.read_series() == a).all()


def test_square_k33_against_table1(stream):
    # the bench workload: k = 33, 16 primes, widths 1..16, autotuned
    primes = gpu_util.seed_primes(16)
    t = golden_io.table1()
    with cp.Sweep("square", 33, primes, stream) as sw:
        assert sw.n_rects == 62 and sw.n_terms == 64
        sw.run()
        sw.sync()
        bulk, surf, corner = sw.series_integers()
        assert bulk == t["alpha"][:64]         # z^0..z^62 exact, z^63 via the mu_32 term
        assert surf == t["beta"][:64]
        assert corner[:63] == t["gamma"][:63]  # the corner series is exact through z^{2k-4}
        pt = sw.read_ptilde()
    # every rectangle: constant term 1 and c_1 = -|E| in all primes
    for (r, s), res in pt.items():
        _, edges = graphs.rectangle_edges("square", r, s)
        for k, p in enumerate(primes):
            assert res[k][0] == 1 and res[k][1] == (-len(edges)) % p
    # sampled rectangles against the plain-C oracle, one prime
    p = primes[0]
    for r in (1, 2, 7, 11):
        hs = [s for rr, s in flm.band(33) if rr == r]
        ref = modp.ptilde_heights("square", r, hs, 63, p)
        for s in hs:
            assert pt[(r, s)][0].tolist() == ref[s].tolist(), (r, s)


def test_triangular_k33_against_baxter_and_printed(stream):
    primes = gpu_util.seed_primes(16)
    tri = golden_io.triangular_series()
    with cp.Sweep("triangular", 33, primes, stream) as sw:
        assert sw.n_terms == 33
        sw.run()
        sw.sync()
        bulk, surf, corner = sw.series_integers()
    assert bulk == flm.baxter_bulk(33)
    assert surf == tri["surface"][:33]
    assert corner == tri["corner"][:33]


def test_sweep_argument_errors(stream):
    primes = gpu_util.seed_primes(4)
    with pytest.raises(cp.CPError):
        cp.Sweep("square", 3, primes, stream)
    with pytest.raises(cp.CPError):
        cp.Sweep("square", 43, primes, stream)
    with pytest.raises(cp.CPError):
        cp.Sweep("square", 12, primes, stream, tile=3, prime_groups=1)
    with pytest.raises(cp.CPError):
        cp.Sweep("square", 12, primes, stream, tile=4, prime_groups=3)
    with pytest.raises(cp.CPError):
        cp.Sweep("square", 12, primes, None, tile=4, prime_groups=1)

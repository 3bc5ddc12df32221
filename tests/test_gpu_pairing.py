"""GPU tests of the two-site tables (cp_set_factor_pairing).

By default the library composes each consecutive pair of square-lattice
per-site factors into one table (T_2 T_1, T_4 T_3, ...; an odd one out stays single), so a row takes
ceil(L/2) launches.  The product is the same matrix, so every result must be
bit-identical to the one-table-per-factor layout of the paper and match the
oracle; widths 1..4 cover the odd-one-out and single-factor chains.
"""
import numpy as np
import pytest

import gpu_util
from oracle import tm_exact

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")


@pytest.fixture(scope="module")
def stream():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()
    return torch.cuda.Stream()


class Pairing:
    def __init__(self, mode):
        self.on = mode

    def __enter__(self):
        self.old = cp.set_factor_pairing(self.on)

    def __exit__(self, *a):
        cp.set_factor_pairing(self.old)


def strip_result(lattice, L, N, primes, D=-1, stream=None):
    with cp.Strip(lattice, L, primes, max_degree=D, max_rows=N, stream=stream) as s:
        s.advance(N - 1)
        return s.read(), s.work()


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_strips_identical_in_both_layouts(lattice, stream):
    for P in (4, 5):  # TMA gather and register gather
        primes = gpu_util.seed_primes(P, seed=8)
        for L, N in [(1, 3), (2, 2), (3, 4), (4, 4), (5, 6), (8, 9), (11, 5)]:
            with Pairing(2):
                a, wa = strip_result(lattice, L, N, primes, stream=stream)
            with Pairing(0):
                b, wb = strip_result(lattice, L, N, primes, stream=stream)
            assert np.array_equal(a, b), (L, N, P)
            if L <= 8:
                assert a.tolist() == gpu_util.residues_of(tm_exact.ptilde(lattice, L, N), primes), (L, N)
            # the same per-site work is counted; the paired layout moves fewer bytes once L >= 2
            assert wa[0] == wb[0] and wa[2] == wb[2]
            if L >= 2 and lattice == "square":  # triangular tables are one per factor in both modes
                # fewer bytes launched; the one-factor-at-a-time figure differs only by the CSR bytes
                assert wa[1] < wb[1]
                if L >= 8:
                    assert abs(wa[4] - wb[1]) < 0.01 * wb[1]
            else:
                assert wa[1] == wb[1] == wa[4] == wb[4]


def test_default_mode_pairs_wide_rows_only(stream):
    assert cp.set_factor_pairing(1) == 1  # the default
    narrow, wide = gpu_util.seed_primes(4), gpu_util.seed_primes(16)
    with cp.Strip("square", 6, narrow, max_degree=20, max_rows=3, stream=stream) as s:  # 21 x 4 words per state
        assert s.work()[1] == s.work()[4]  # one table per factor
    with cp.Strip("square", 6, wide, max_degree=63, max_rows=3, stream=stream) as s:  # 64 x 16 words: 4 KB
        assert s.work()[1] < s.work()[4]  # two-site tables


@pytest.mark.parametrize("lattice,k", [("square", 17), ("triangular", 14)])
def test_sweeps_identical_in_both_layouts(lattice, k, stream):
    primes = gpu_util.seed_primes(8, seed=6)
    out = []
    for on in (2, 0):
        with Pairing(on):
            with cp.Sweep(lattice, k, primes, stream, tile=4, prime_groups=1) as sw:
                sw.run()
                sw.sync()
                out.append((sw.read_series(), sw.read_ptilde(), sw.updates_per_run, sw.bytes_per_run,
                            sw.launches_per_run))
    (sa, pa, ua, ba, la), (sb, pb, ub, bb, lb) = out
    assert np.array_equal(sa, sb)
    assert pa.keys() == pb.keys() and all(np.array_equal(pa[x], pb[x]) for x in pa)
    assert ua == ub
    if lattice == "square":
        assert ba < bb and la < lb
    else:
        assert ba == bb and la == lb


def test_server_identical_in_both_layouts(stream):
    reqs = [("square", 7, 8, gpu_util.seed_primes(4, seed=1)), ("triangular", 6, 6, gpu_util.seed_primes(5, seed=2)),
            ("square", 3, 3, gpu_util.seed_primes(3, seed=3))]
    got = {}
    for on in (2, 0):
        with Pairing(on):
            with cp.Server(1 << 28, max_active=8, stream=stream) as sv:
                ids = [sv.submit(*r) for r in reqs]
                while any(sv.result(i)[0] != sv.DONE for i in ids):
                    sv.step()
                got[on] = [sv.result(i)[1] for i in ids]
    for a, b, r in zip(got[2], got[0], reqs):
        assert np.array_equal(a, b)
        assert a.tolist() == gpu_util.residues_of(tm_exact.ptilde(r[0], r[1], r[2]), r[3])

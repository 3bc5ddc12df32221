"""Per-rectangle parity at the production widths.

The k = 33 sweeps (square: D = 63, rows of 4 KB with two-site tables;
triangular: D = 32, rows of 2.1 KB) run their widest strips through the TMA
gather.  Every band rectangle of widths 12, 13 and 14 is compared element by
element with the plain-C mod-p oracle on 4 of the sweep's 16 primes, and a
width-14 full-degree request (16 primes, rows of 13 KB split into column
tasks) goes through the server and is compared on 2 primes.  The oracle runs
in a spawn process pool while the GPU works.
"""
import multiprocessing as mp

import pytest

import gpu_util
from oracle import flm

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")

WIDTHS = (12, 13, 14)
PRIME_IDX = (0, 5, 10, 15)
K = 33


def _oracle_strip(args):
    lattice, r, heights, D, p = args
    from oracle import modp
    return {s: v.tolist() for s, v in modp.ptilde_heights(lattice, r, heights, D, p).items()}


@pytest.fixture(scope="module")
def oracle_jobs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    primes = gpu_util.seed_primes(16)
    pool = mp.get_context("spawn").Pool(16)
    jobs = {}
    for lattice in ("square", "triangular"):
        D = flm.n_terms(lattice, K) + (1 if lattice == "square" and K % 2 else 0) - 1
        for r in WIDTHS:
            hs = [s for rr, s in flm.band(K) if rr == r]
            for i in PRIME_IDX:
                jobs[(lattice, r, i)] = pool.apply_async(_oracle_strip, ((lattice, r, hs, D, primes[i]),))
    sp = gpu_util.seed_primes(16, seed=9)
    for i in (0, 15):
        jobs[("server", 14, i)] = pool.apply_async(_oracle_strip, (("square", 14, [15], 14 * 15 - 1, sp[i]),))
    yield primes, sp, jobs
    pool.terminate()


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_sweep_widths_12_to_14_against_oracle(oracle_jobs, lattice):
    import torch
    primes, _, jobs = oracle_jobs
    stream = torch.cuda.Stream()
    with cp.Sweep(lattice, K, primes, stream) as sw:  # production path: autotuned tile and grouping
        sw.run()
        sw.sync()
        pt = sw.read_ptilde()
        n = sw.n_terms
    for r in WIDTHS:
        for i in PRIME_IDX:
            ref = jobs[(lattice, r, i)].get(timeout=900)
            for s, want in ref.items():
                assert pt[(r, s)][i].tolist() == want[:n], (lattice, r, s, i)


def test_server_width14_full_degree_sixteen_primes(oracle_jobs):
    import torch
    _, sp, jobs = oracle_jobs
    stream = torch.cuda.Stream()
    with cp.Server(64 << 30, max_active=4, stream=stream) as sv:
        rid = sv.submit("square", 14, 15, sp)
        small = sv.submit("triangular", 5, 6, sp[:4])  # in the mix with it
        while sv.result(rid)[0] != sv.DONE or sv.result(small)[0] != sv.DONE:
            sv.step()
        _, got, _ = sv.result(rid)
    for i in (0, 15):
        assert got[i].tolist() == jobs[("server", 14, i)].get(timeout=900)[15], i

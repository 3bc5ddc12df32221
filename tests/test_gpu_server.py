"""GPU tests of the continuous-batching server (cp_server_*).

Every result is compared bit-exactly with the oracle, and with the same request
served alone; admission by memory is exercised with a budget that holds only a
few requests at once, with requests arriving while others are on the GPU.
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


def mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        lattice = "square" if rng.integers(0, 2) == 0 else "triangular"
        L = int(rng.integers(1, 8))
        N = L + int(rng.integers(0, 2))
        P = int(rng.choice([1, 3, 4, 5, 8]))
        out.append((lattice, L, N, gpu_util.seed_primes(P, seed=100 + j)))
    return out


def run_all(server, reqs, arrivals_per_step=None):
    ids = []
    pending = list(reqs)
    while pending or any(server.result(i)[0] != server.DONE for i in ids):
        take = len(pending) if arrivals_per_step is None else arrivals_per_step
        for r in pending[:take]:
            ids.append(server.submit(*r))
        pending = pending[take:]
        server.step()
    return [server.result(i)[1] for i in ids]


def test_mixed_stream_matches_oracle_and_alone(stream):
    reqs = mixed_requests(24, seed=5)
    with cp.Server(1 << 30, max_active=64, stream=stream) as sv:
        mixed = run_all(sv, reqs, arrivals_per_step=3)  # requests arrive while others run
        assert sv.stats()["arena_free_bytes"] == 1 << 30
    for (lattice, L, N, primes), got in zip(reqs, mixed):
        want = tm_exact.ptilde(lattice, L, N)
        assert got.tolist() == gpu_util.residues_of(want, primes), (lattice, L, N, len(primes))
    # each request alone on a fresh server gives the same residues
    for r, got in zip(reqs[:8], mixed[:8]):
        with cp.Server(1 << 28, max_active=1, stream=stream) as sv:
            alone = run_all(sv, [r])[0]
        assert np.array_equal(alone, got)
        with cp.Strip(r[0], r[1], r[3], max_degree=-1, max_rows=r[2], stream=stream) as s:
            s.advance(r[2] - 1)
            assert np.array_equal(s.read(), got)


def test_admission_by_memory(stream):
    # 12 requests of width 9 (~2.8 MB each with 8 primes); an 8 MB budget holds 2 at a time
    reqs = [("square", 9, 9, gpu_util.seed_primes(8, seed=200 + j)) for j in range(12)]
    with cp.Server(8 << 20, max_active=64, stream=stream) as sv:
        ids = [sv.submit(*r) for r in reqs]
        peak_active, saw_queue = 0, False
        while any(sv.result(i)[0] != sv.DONE for i in ids):
            a, q, _ = sv.step()
            peak_active = max(peak_active, a)
            saw_queue = saw_queue or q > 0
        assert saw_queue and 1 <= peak_active < len(reqs)
        assert sv.stats()["arena_free_bytes"] == 8 << 20
        want = tm_exact.ptilde("square", 9, 9)
        for r, i in zip(reqs, ids):
            st, got, (t_sub, t_adm, t_done) = sv.result(i)
            assert st == sv.DONE and t_sub <= t_adm <= t_done
            assert got.tolist() == gpu_util.residues_of(want, r[3])


def test_oversize_request_rejected(stream):
    with cp.Server(4 << 20, max_active=4, stream=stream) as sv:
        with pytest.raises(cp.CPError):
            sv.submit("square", 12, 12, gpu_util.seed_primes(8))
        # a small one still runs
        rid = sv.submit("triangular", 3, 3, gpu_util.seed_primes(2))
        while sv.result(rid)[0] != sv.DONE:
            sv.step()


def test_same_rectangle_requests_merge(stream):
    # requests for one rectangle with assorted prime counts share jobs; each gets its own residues
    counts = [1, 3, 5, 7, 2, 4, 6, 9]
    reqs = [("triangular", 6, 7, gpu_util.seed_primes(c, seed=300 + j)) for j, c in enumerate(counts)]
    with cp.Server(1 << 28, max_active=8, stream=stream) as sv:
        got = run_all(sv, reqs)
        steps = sv.stats()["steps"]
    want = tm_exact.ptilde("triangular", 6, 7)
    for r, g in zip(reqs, got):
        assert g.tolist() == gpu_util.residues_of(want, r[3])
    # merged: far fewer steps than one job per request would need if run one after another
    assert steps < 2 * (6 * 6 + 5 + 1)

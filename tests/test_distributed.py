"""Sharding by primes across ranks (world size 2, gloo, CPU): the gathered residues
of both ranks recombine to the exact series.  The per-rank compute is done by the
oracle here (no GPU); the host plumbing is the library's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import synthetic_inputs
    from oracle import crt, flm, tm_exact
    from paper_1005_3609_gb300 import distributed as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    all_primes = crt.primes_from_draws(synthetic_inputs.prime_draws(0, 64), 6)
    lo, hi = D.rank_prime_slice(len(all_primes), world, rank)
    mine = all_primes[lo:hi]
    k, n = 13, 13
    pt = {}
    for r in range(1, k // 2 + 1):
        hs = [s for rr, s in flm.band(k) if rr == r]
        got = tm_exact.ptilde_heights("triangular", r, hs, n - 1)
        pt.update({(r, s): got[s] for s in hs})
    series = flm.flm_series("triangular", k, pt, n)
    res = np.array([[[c % p for c in series[x]] for p in mine] for x in range(3)], dtype=np.uint32)
    out = D.gather_residues(res, mine, dist)
    if rank == 0:
        res_all, primes_all = out
        assert primes_all == all_primes
        got = [crt.crt_signed(res_all[x].tolist(), primes_all) for x in range(3)]
        q.put(got == [list(s) for s in series] and got[0] == flm.baxter_bulk(n))
    else:
        assert out is None
    dist.barrier()
    dist.destroy_process_group()


def test_rank_prime_slices_partition():
    from paper_1005_3609_gb300 import distributed as D
    for n in range(1, 40):
        for w in range(1, 9):
            cover = []
            for r in range(w):
                lo, hi = D.rank_prime_slice(n, w, r)
                cover += list(range(lo, hi))
            assert cover == list(range(n))


def test_two_rank_gather_and_crt():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True

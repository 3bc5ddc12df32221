"""Multi-GPU sharding of the sweep by primes (host logic).

The residue computations of different primes are independent (Sec. 3.5), so
ranks never exchange data while they compute: each rank sweeps its own primes
on its own GPU.  The one exchange is at the end, when rank 0 gathers every
rank's series residues and primes for the Chinese remaindering.
"""
import numpy as np


def rank_prime_slice(n_total, world, rank):
    """Contiguous block of prime indices of `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_residues(residues, primes, dist, dst=0):
    """residues: uint32 [3][P_local][n]; primes: P_local ints.
    On `dst` returns (uint32 [3][P_total][n], primes in rank order); elsewhere None."""
    payload = (np.ascontiguousarray(residues, dtype=np.uint32), [int(p) for p in primes])
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(payload, out, dst=dst)
    if out is None:
        return None
    res = np.concatenate([r for r, _ in out], axis=1)
    prs = [p for _, ps in out for p in ps]
    if len(set(prs)) != len(prs):
        raise ValueError("ranks swept overlapping primes")
    return res, prs

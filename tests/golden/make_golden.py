"""Write the exact P~ coefficients of the fixed rectangles into tests/golden/.

Run from the repository root:  python tests/golden/make_golden.py
Uses only ``oracle/`` and the seeded prime draws of ``synthetic_inputs``.

* square 5 x 6: exact Python-integer transfer matrix (oracle.tm_exact);
* square 12 x 13 and triangular 13 x 14: the plain-C mod-p oracle for the
  seed-0 primes, recombined by CRT (Sec. 3.5).  Primes are added until the
  product exceeds twice Whitney's bound max_j C(|E|, j) >= |c_j| and the result
  no longer changes when two more primes are added (the paper's stabilisation
  rule).
"""
import multiprocessing as mp
import os
import sys
from math import comb

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import crt, graphs, modp, tm_exact  # noqa: E402
import synthetic_inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _residues(args):
    lattice, L, N, p = args
    return [int(x) for x in modp.ptilde(lattice, L, N, L * N - 1, p)]


def exact_by_crt(lattice, L, N, pool):
    nv, edges = graphs.rectangle_edges(lattice, L, N)
    bound = max(comb(len(edges), j) for j in range(nv))
    primes = crt.primes_from_draws(synthetic_inputs.prime_draws(0, 256), 64)
    need = 1
    prod = 1
    while prod <= 2 * bound:
        prod *= primes[need - 1]
        need += 1
    use = primes[: need + 2]
    rows = pool.map(_residues, [(lattice, L, N, p) for p in use])
    full = crt.crt_signed(rows, use)
    assert crt.crt_signed(rows[:-2], use[:-2]) == full, "CRT did not stabilise"
    return full, use


def write(name, lattice, L, N, coeffs, how):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# P~ = q^{-|V|} P(q) = sum_j c_j w^j (w = 1/q) of the %s-lattice %d x %d rectangle\n" % (lattice, L, N))
        f.write("# (L = %d sites per row, N = %d rows, free boundaries), exact integers.\n" % (L, N))
        f.write("# Written by tests/golden/make_golden.py: %s\n" % how)
        f.write("# j c_j\n")
        for j, c in enumerate(coeffs):
            f.write("%d %d\n" % (j, c))


def main():
    c1 = tm_exact.ptilde("square", 5, 6)
    write("ptilde_square_5x6.txt", "square", 5, 6, c1, "oracle.tm_exact (exact integers)")
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(os.cpu_count() or 1, 18)) as pool:
        for lattice, L, N in [("square", 12, 13), ("triangular", 13, 14)]:
            full, use = exact_by_crt(lattice, L, N, pool)
            write("ptilde_%s_%dx%d.txt" % (lattice, L, N), lattice, L, N, full,
                  "oracle.modp residues for %d seed-0 primes, CRT (stable under the last two)" % len(use))
            print(lattice, L, N, "primes", len(use))


if __name__ == "__main__":
    main()

"""A small, fixed invocation of the strip path for profilers (ncu).

python -m paper_1005_3609_gb300.profile_case --lattice square --L 14 --D 63 --primes 16 --rows 1

Builds the tables, then advances one strip by `rows` rows (one gather launch
per table of the row: L per-site tables, or ceil(L/2) two-site tables with
--pairing 2 or, for square rows of 3 KB or more, the default --pairing 1) and
reads P~ once.  Prints the launch count.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="square")
    ap.add_argument("--L", type=int, default=14)
    ap.add_argument("--D", type=int, default=63)
    ap.add_argument("--primes", type=int, default=16)
    ap.add_argument("--rows", type=int, default=1)
    ap.add_argument("--pairing", type=int, default=1, help="table layout (cp_set_factor_pairing)")
    a = ap.parse_args()
    import synthetic_inputs
    import paper_1005_3609_gb300 as cp
    primes = cp.select_primes(synthetic_inputs.prime_draws(0, 64), a.primes)
    cp.set_factor_pairing(a.pairing)
    with cp.Strip(a.lattice, a.L, primes, max_degree=a.D, max_rows=a.rows + 2) as s:
        s.advance(1)  # warm-up row
        s.advance(a.rows)
        s.read()
        w = s.work()
        per_row = (a.L + 1) // 2 if w[1] < w[4] else a.L
        readout = max(1, a.L // 2 if w[1] < w[4] else a.L - 1)
        print("states", s.n_states, "gather launches per row", per_row,
              "total", per_row * (a.rows + 1) + readout)


if __name__ == "__main__":
    main()

"""Helpers of the GPU tests: primes from the seeded draws and closed forms."""
import synthetic_inputs
from oracle import crt as ocrt


def seed_primes(n, seed=0):
    return ocrt.primes_from_draws(synthetic_inputs.prime_draws(seed, 256), n)


def residues_of(coeffs, primes):
    return [[c % p for c in coeffs] for p in primes]


def ptilde_of_q_product(factors, nv):
    """P~ coefficients of a product of polynomials in q (ascending lists)."""
    out = [1]
    for f in factors:
        nxt = [0] * (len(out) + len(f) - 1)
        for i, a in enumerate(out):
            for j, b in enumerate(f):
                nxt[i + j] += a * b
        out = nxt
    out += [0] * (nv + 1 - len(out))
    return [out[nv - j] for j in range(nv)]

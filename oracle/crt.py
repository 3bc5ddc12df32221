"""Primes and Chinese remaindering (Sec. 3.5).

Test infrastructure only (see ``oracle/__init__``).

The paper computes P~ modulo several primes p < 2^31 held in 32-bit words and
recombines them by the Chinese remainder theorem, adding primes until the
result stops changing.  It does not say how the primes were chosen; the
reading used throughout is: take raw draws r_k in [2^30, 2^31) from a seeded
generator, map each to the smallest prime >= r_k, drop repeats, keep the
first n.  Primality here is trial division (plain, obviously correct).
"""


def is_prime(n):
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def primes_from_draws(draws, n):
    out = []
    for r in draws:
        p = int(r)
        while not is_prime(p):
            p += 1
        if p >= 1 << 31:
            continue
        if p not in out:
            out.append(p)
        if len(out) == n:
            return out
    raise ValueError("not enough draws for %d primes" % n)


def crt(residues, primes):
    """Smallest non-negative x with x = r_i mod p_i (iterative, exact)."""
    x, mod = 0, 1
    for r, p in zip(residues, primes):
        # x + mod * t = r (mod p)
        t = ((r - x) * pow(mod, -1, p)) % p
        x += mod * t
        mod *= p
    return x, mod


def symmetric(x, mod):
    return x - mod if x > mod // 2 else x


def crt_signed(residue_rows, primes):
    """residue_rows[k][j] = c_j mod primes[k] -> list of signed c_j."""
    n = len(residue_rows[0])
    out = []
    for j in range(n):
        x, mod = crt([row[j] for row in residue_rows], primes)
        out.append(symmetric(x, mod))
    return out

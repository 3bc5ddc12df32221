"""Chromatic polynomial from its definition: count proper q-colourings (Sec. 1).

Test infrastructure only (see ``oracle/__init__``).

P_G(q) is the number of colourings of the vertices with q colours such that
adjacent vertices differ.  It is a polynomial of degree |V|, so its values at
q = 0..|V| determine it; the coefficients follow from Newton's forward
differences, in exact rational arithmetic.

Colourings are counted on the rectangle row by row, keeping the colours of the
last L vertices (a sliding window), which is only a way of enumerating all
colourings without listing them one by one.  The adjacency used here is
written out from the lattice description and is NOT taken from
``oracle.graphs``, so the two cross-check each other.
"""
from fractions import Fraction


def count_colourings(lattice, L, N, q):
    """Number of proper q-colourings of the L x N rectangle (exact)."""
    if q == 0:
        return 0
    # window holds the colours of the previous L vertices in row-major order:
    # for vertex (t, i) these are (t-1, i), (t-1, i+1), ..., (t-1, L-1), (t, 0), ..., (t, i-1)
    states = {(): 1}
    for t in range(N):
        for i in range(L):
            new = {}
            for win, cnt in states.items():
                for c in range(q):
                    if i >= 1 and win[-1] == c:  # left neighbour (t, i-1)
                        continue
                    if t >= 1:
                        if win[-L] == c:  # up neighbour (t-1, i)
                            continue
                        # triangular: (t-1, i+1) is joined to (t, i)
                        if lattice == "triangular" and i + 1 < L and win[-L + 1] == c:
                            continue
                    w2 = (win + (c,))[-L:]
                    new[w2] = new.get(w2, 0) + cnt
            states = new
    return sum(states.values())


def poly_from_values(values):
    """Coefficients (ascending powers of q) of the degree-len(values)-1 polynomial
    taking values[k] at q = k, by Newton forward differences."""
    n = len(values)
    diffs = [Fraction(v) for v in values]
    newton = []
    for _ in range(n):
        newton.append(diffs[0])
        diffs = [diffs[j + 1] - diffs[j] for j in range(len(diffs) - 1)]
    # P(q) = sum_k newton[k] * binom(q, k) ; expand binom(q, k) = q(q-1)...(q-k+1)/k!
    coeffs = [Fraction(0)] * n
    falling = [Fraction(1)]  # coefficients of q(q-1)...(q-k+1)
    fact = 1
    for k in range(n):
        if k > 0:
            fact *= k
            nxt = [Fraction(0)] * (len(falling) + 1)
            for p, c in enumerate(falling):
                nxt[p + 1] += c
                nxt[p] -= c * (k - 1)
            falling = nxt
        for p, c in enumerate(falling):
            coeffs[p] += newton[k] * c / fact
    out = []
    for c in coeffs:
        if c.denominator != 1:
            raise ArithmeticError("non-integer coefficient")
        out.append(int(c))
    return out


def chromatic_poly(lattice, L, N):
    """Coefficients of P_G(q), ascending powers of q, for the L x N rectangle."""
    nv = L * N
    return poly_from_values([count_colourings(lattice, L, N, q) for q in range(nv + 1)])

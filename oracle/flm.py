"""Finite-lattice method and the series checks (Sec. 4.1-4.3), exact integers.

Test infrastructure only (see ``oracle/__init__``).

Series are lists of Python ints, index = power, truncated to `n` terms.

* Expansion variables: z = 1/(q-1) on the square lattice, eq. (def_z), so
  w = 1/q = z/(1+z); x with q = 2 - x - 1/x on the triangular lattice (Sec. 4.3),
  so w = -x/(1-x)^2.
* f_b, f_s, f_c = log q (f_b only) + sum over B(k) of weight * log P~_{r,s},
  eqs. (fb)-(fc).  Exponentiating turns the sums of logarithms into products
  of integer powers, E = prod P~_{r,s}^{weight}, which needs no logarithm and
  no rational number because every P~ has constant term 1 (Sec. 3.5).
* Table 1 gives exp(f_b) = (q-1)^2/q sum alpha_k z^k, so sum alpha_k z^k =
  (1+z)^2 E_b; exp(f_s) = E_s; exp(f_c) = E_c.
* Triangular bulk: exp(f_b) = q E_b = -(1-x)^2/x E_b, and Baxter's product,
  eq. (efb), gives exp(f_b) = -(1/x) prod(...), so (1-x)^2 E_b = prod(...).

Reading of the surface weight (Sec. 4.1): the printed coefficient of
delta_{r+s,k-3} in beta_k, (r+s-2)/2, violates the sum rules that
log P = mn f_b + (m+n) f_s + f_c imposes (sum beta*rs = 0, sum beta*(r+s) = 1,
sum beta = 0); (r+s+2)/2 is the unique linear coefficient that satisfies them
and reproduces Table 1.  `beta` uses it; `beta_printed` keeps the printed form
for the test that shows it fails.
B(k) includes the 1 x s strips (r = 1).
"""
from fractions import Fraction
from math import comb


# ---------------------------------------------------------------- series ops

def mul(a, b, n):
    out = [0] * n
    for i, x in enumerate(a[:n]):
        if x == 0:
            continue
        for j in range(min(len(b), n - i)):
            out[i + j] += x * b[j]
    return out


def inverse(a, n):
    assert a[0] in (1, -1)
    b = [0] * n
    b[0] = a[0]  # 1/a0 == a0 for a0 = +-1
    for k in range(1, n):
        acc = 0
        for i in range(1, min(k, len(a) - 1) + 1):
            acc += a[i] * b[k - i]
        b[k] = -acc * a[0]
    return b


def power(a, e, n):
    if e < 0:
        a, e = inverse(a, n), -e
    out = [1] + [0] * (n - 1)
    base = list(a[:n]) + [0] * max(0, n - len(a))
    while e:
        if e & 1:
            out = mul(out, base, n)
        base = mul(base, base, n)
        e >>= 1
    return out


def compose_w(ptilde, wseries, n):
    """P~(w(t)) for a series w(t) without constant term, by Horner's rule."""
    out = [0] * n
    for c in reversed(ptilde):
        out = mul(out, wseries, n)
        out[0] += c
    return out


def w_of_z(n):
    """w = z/(1+z) = z - z^2 + z^3 - ..."""
    return [0] + [(-1) ** (i + 1) for i in range(1, n)]


def w_of_x(n):
    """w = -x/(1-x)^2 = -(x + 2x^2 + 3x^3 + ...)."""
    return [0] + [-i for i in range(1, n)]


# ---------------------------------------------------------------- weights

def _d(a, b):
    return 1 if a == b else 0


def alpha(k, r, s):
    t = r + s
    return (2 - _d(r, s)) * (_d(t, k) - 3 * _d(t, k - 1) + 3 * _d(t, k - 2) - _d(t, k - 3))


def _beta(k, r, s, last):
    t = r + s
    v = (2 - _d(r, s)) * (Fraction(2 - t, 2) * _d(t, k) + Fraction(3 * t - 2, 2) * _d(t, k - 1)
                          - Fraction(3 * t + 2, 2) * _d(t, k - 2) + last(t) * _d(t, k - 3))
    return v


def beta(k, r, s):
    v = _beta(k, r, s, lambda t: Fraction(t + 2, 2))
    assert v.denominator == 1
    return int(v)


def beta_printed(k, r, s):
    return _beta(k, r, s, lambda t: Fraction(t - 2, 2))


def gamma(k, r, s):
    t = r + s
    return (2 - _d(r, s)) * ((r - 1) * (s - 1) * _d(t, k) + (1 + t - 3 * r * s) * _d(t, k - 1)
                             + (3 * r * s + t - 1) * _d(t, k - 2) - (r + 1) * (s + 1) * _d(t, k - 3))


def band(k):
    """Rectangles (r, s), r <= s, r >= 1, with a non-zero weight: k-3 <= r+s <= k."""
    return [(r, s) for r in range(1, k + 1) for s in range(r, k + 1) if k - 3 <= r + s <= k]


def n_terms(lattice, k):
    """Series length fixed by the error terms: O(z^{2k-3}) square, O(x^k) triangular."""
    return 2 * k - 3 if lattice == "square" else k


# ---------------------------------------------------------------- series

def flm_series(lattice, k, ptildes, n=None):
    """ptildes[(r, s)] = coefficients of P~ in w (any truncation >= n-1).
    Returns (bulk, surface, corner): square -> (sum alpha z^k, E_s, E_c);
    triangular -> ((1-x)^2 E_b, E_s, E_c)."""
    if n is None:
        n = n_terms(lattice, k)
    ws = w_of_z(n) if lattice == "square" else w_of_x(n)
    eb = [1] + [0] * (n - 1)
    es = list(eb)
    ec = list(eb)
    for (r, s) in band(k):
        p = compose_w(list(ptildes[(r, s)])[:n], ws, n)
        eb = mul(eb, power(p, alpha(k, r, s), n), n)
        es = mul(es, power(p, beta(k, r, s), n), n)
        ec = mul(ec, power(p, gamma(k, r, s), n), n)
    pref = [1, 2, 1] if lattice == "square" else [1, -2, 1]
    return mul(pref, eb, n), es, ec


def mu_series(pmax):
    """mu_p for p = 0..pmax from the generating function of Sec. 4.2 (y = x^2)."""
    n = pmax + 1
    cat = [comb(2 * j, j) // (j + 1) for j in range(n + 1)]
    sq = [Fraction(1)] + [Fraction(-2 * cat[j - 1]) for j in range(1, n)]  # sqrt(1-4y)
    one4 = [Fraction(4) ** j for j in range(n)]                              # 1/(1-4y)

    def fmul(a, b):
        out = [Fraction(0)] * n
        for i in range(n):
            for j in range(n - i):
                out[i + j] += a[i] * b[j]
        return out

    inv2y = [Fraction((-1) ** j, 2 ** (j + 1)) for j in range(n)]           # 1/(2+y)
    num1 = [Fraction(0)] * n
    num1[0] += 2
    if n > 1:
        num1[1] -= 2
    ysq = [Fraction(0)] + sq[: n - 1]
    num1 = [a - b for a, b in zip(num1, ysq)]
    t1 = fmul(fmul(num1, one4), inv2y)
    num2 = [Fraction(0)] * n
    num2[0] += 3
    if n > 1:
        num2[1] -= 4
    num2 = [a - 4 * b for a, b in zip(num2, sq)]
    t2 = fmul(num2, fmul(one4, one4))
    out = [Fraction(0)] * n
    for p in range(n):
        if p >= 4:
            out[p] += t1[p - 4]
        if p >= 6:
            out[p] += t2[p - 6]
    assert all(x.denominator == 1 for x in out)
    return [int(x) for x in out]


def _product(factors, n):
    """prod over (exponent e, power a) of (1 - x^a)^e, truncated to n terms."""
    out = [1] + [0] * (n - 1)
    for e, a in factors:
        if a >= n or e == 0:
            continue
        f = [0] * n
        f[0] = 1
        f[a] = -1
        out = mul(out, power(f, e, n), n)
    return out


def baxter_bulk(n):
    """prod_j (1-x^{6j-3})(1-x^{6j-2})^2(1-x^{6j-1}) / [(1-x^{6j-5})(1-x^{6j-4})(1-x^{6j})(1-x^{6j+1})], eq. (efb)."""
    fac = []
    for j in range(1, n // 6 + 2):
        fac += [(1, 6 * j - 3), (2, 6 * j - 2), (1, 6 * j - 1),
                (-1, 6 * j - 5), (-1, 6 * j - 4), (-1, 6 * j), (-1, 6 * j + 1)]
    return _product(fac, n)


def conjectured_surface(n):
    """Eq. (efs)."""
    fac = []
    for j in range(1, n // 12 + 2):
        fac += [(2, 12 * j - 11), (2, 12 * j - 6), (2, 12 * j - 5), (2, 12 * j - 4),
                (-2, 12 * j - 9), (-2, 12 * j - 8), (-2, 12 * j - 7), (-2, 12 * j - 2)]
    return _product(fac, n)


def conjectured_corner(n):
    """Eq. (efc)."""
    ex = {11: -1, 10: 1, 9: 3, 8: 2, 7: 4, 6: -3, 5: 1, 4: -3, 3: 5, 2: 2, 1: 2, 0: 1}
    fac = []
    for j in range(1, n // 12 + 2):
        fac += [(e, 12 * j - kk) for kk, e in ex.items()]
    return _product(fac, n)

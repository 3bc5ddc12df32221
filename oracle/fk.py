"""Fortuin-Kasteleyn subset expansion, eqs. (Z2) and (Z_modified), Sec. 2 and 3.1.

Test infrastructure only (see ``oracle/__init__``).

Z~_G(q, v) = sum over edge subsets A of q^{k(A) - |V|} v^{|A|}, with k(A) the
number of connected components of (V, A).  In w = 1/q this is a polynomial
whose coefficient of w^j collects the subsets with |V| - k(A) = j.  The
chromatic polynomial is the special case v = -1.  Brute force over all 2^|E|
subsets, so only for tiny graphs.
"""


def _components(n, edges):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    k = n
    for u, v in edges:
        a, b = find(u), find(v)
        if a != b:
            parent[a] = b
            k -= 1
    return k


def ztilde(n, edges, v):
    """Coefficients of Z~ in w (ascending), for an integer v."""
    m = len(edges)
    out = [0] * n
    for mask in range(1 << m):
        sub = [edges[b] for b in range(m) if mask >> b & 1]
        j = n - _components(n, sub)
        out[j] += v ** len(sub)
    return out

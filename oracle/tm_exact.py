"""The paper's sparse projected transfer matrix, exact integers (Sec. 3.1-3.3).

Test infrastructure only (see ``oracle/__init__``).

A vector is a dict {partition tuple: [c_0, ..., c_D]} holding, for each
connectivity state, a polynomial in w = 1/q truncated after w^D (Sec. 3.5).
Every operator is applied literally, one single-edge operator at a time, on
the hash map (the "standard hashing" alternative of Sec. 3.4; no ranks):

* J_{a,b}: identity if a, b share a block, else join their blocks with a
  factor w (Sec. 3.1);
* H_{a,b} = 1 + v J_{a,b} (Sec. 3.1), here at v = -1 unless stated;
* D_i: make site i a singleton (Sec. 3.1);
* V_i = v w + D_i (Sec. 3.1);
* P_{a,b}: keep a state iff a, b are in different blocks, eq. (projector).

Square lattice, eqs. (T_sq_decomp), (T_sq_proj):
  T = T_m ... T_1, T_i = (prod_{j != i} P_{j,j+1}) V_i H_{i,i+1} (i < m),
  T_m = (prod_j P_{j,j+1}) V_m.
Triangular lattice (Sec. 3.3):
  T_i = (prod_j P_{j,j+1}) V_i H_{i-1,i} H_{i,i+1}, the missing H dropped at
  i = 1 and i = m.
Last row, eqs. (T_last), (T_last_i), both lattices:
  T_i^last = (prod_{j>i} P_{j,j+1}) D_i H_{i,i+1}; for i = m the factor
  H_{m,m+1} does not exist and T_m^last = D_m.
P~ = coefficient of e_0 in T_last T^{n-1} e_0, eq. (Z_from_T).

Sites are 0-based in code (the paper's site i is index i-1).
"""
from .partitions import canon


def _acc(out, s, poly, coef, shift, D):
    if coef == 0:
        return
    tgt = out.get(s)
    if tgt is None:
        tgt = [0] * (D + 1)
        out[s] = tgt
    for j in range(D + 1 - shift):
        tgt[j + shift] += coef * poly[j]


def _clean(out):
    return {s: p for s, p in out.items() if any(p)}


def join(s, a, b):
    """J_{a,b} on one partition: (new partition, power of w)."""
    if s[a] == s[b]:
        return s, 0
    la, lb = s[a], s[b]
    return canon(tuple(la if x == lb else x for x in s)), 1


def detach(s, i):
    """D_i on one partition."""
    fresh = max(s) + 1
    lab = list(s)
    lab[i] = fresh
    return canon(lab)


def op_H(vec, a, b, D, v=-1):
    out = {}
    for s, p in vec.items():
        _acc(out, s, p, 1, 0, D)
        t, k = join(s, a, b)
        _acc(out, t, p, v, k, D)
    return _clean(out)


def op_D(vec, i, D):
    out = {}
    for s, p in vec.items():
        _acc(out, detach(s, i), p, 1, 0, D)
    return _clean(out)


def op_V(vec, i, D, v=-1):
    out = {}
    for s, p in vec.items():
        _acc(out, detach(s, i), p, 1, 0, D)
        _acc(out, s, p, v, 1, D)
    return _clean(out)


def op_P(vec, a, b):
    return {s: p for s, p in vec.items() if s[a] != s[b]}


def site_op(lattice, m, i, vec, D):
    """The per-site factor T_i (0-based i) of one row."""
    if lattice == "square":
        if i < m - 1:
            vec = op_H(vec, i, i + 1, D)
        vec = op_V(vec, i, D)
        for j in range(m - 1):
            if j != i or i == m - 1:
                vec = op_P(vec, j, j + 1)
        return vec
    if lattice == "triangular":
        if i < m - 1:
            vec = op_H(vec, i, i + 1, D)
        if i > 0:
            vec = op_H(vec, i - 1, i, D)
        vec = op_V(vec, i, D)
        for j in range(m - 1):
            vec = op_P(vec, j, j + 1)
        return vec
    raise ValueError(lattice)


def last_op(m, i, vec, D):
    """T_i^last (0-based i), eq. (T_last_i); identical for both lattices."""
    if i < m - 1:
        vec = op_H(vec, i, i + 1, D)
    vec = op_D(vec, i, D)
    for j in range(i + 1, m - 1):
        vec = op_P(vec, j, j + 1)
    return vec


def e0(m, D):
    return {tuple(range(m)): [1] + [0] * D}


def advance(lattice, m, vec, n_rows, D):
    for _ in range(n_rows):
        for i in range(m):
            vec = site_op(lattice, m, i, vec, D)
    return vec


def readout(m, vec, D):
    for i in range(m):
        vec = last_op(m, i, vec, D)
    assert set(vec) <= {tuple(range(m))}
    return list(vec.get(tuple(range(m)), [0] * (D + 1)))


def ptilde(lattice, L, N, D=None):
    """Coefficients c_0..c_D of P~ = q^{-LN} P(q) in w = 1/q for the L x N
    rectangle (L sites per row, N rows); D defaults to the full degree LN-1."""
    if D is None:
        D = L * N - 1
    vec = advance(lattice, L, e0(L, D), N - 1, D)
    return readout(L, vec, D)


def ptilde_heights(lattice, L, heights, D):
    """P~ of L x s for every s in `heights`, from one strip (same row operator)."""
    out = {}
    vec = e0(L, D)
    h = 1
    for s in sorted(heights):
        vec = advance(lattice, L, vec, s - h, D)
        h = s
        out[s] = readout(L, vec, D)
    return out

"""Rectangles of the square and triangular lattices with free boundaries.

Test infrastructure only (see ``oracle/__init__``).

A rectangle of width L (vertices per row, the strip width m of Sec. 3) and
height N (rows) has vertex (t, i) = row t in 0..N-1, column i in 0..L-1,
numbered t*L + i.  The square lattice has the horizontal edges (t,i)-(t,i+1)
and the vertical edges (t,i)-(t+1,i).  The triangular lattice is the square
lattice with one diagonal per face, all in the same orientation (Sec. 3.3):
the transfer matrix lays H_{i-1,i} after site i-1 has moved up a row and
before site i has, so the diagonal joins (t, i) to (t+1, i-1).
"""

SQUARE = "square"
TRIANGULAR = "triangular"


def rectangle_edges(lattice, L, N):
    """Return (number of vertices, list of edges (u, v) with u < v)."""
    if lattice not in (SQUARE, TRIANGULAR):
        raise ValueError(lattice)
    if L < 1 or N < 1:
        raise ValueError("empty rectangle")
    edges = []
    vid = lambda t, i: t * L + i
    for t in range(N):
        for i in range(L):
            if i + 1 < L:
                edges.append((vid(t, i), vid(t, i + 1)))
            if t + 1 < N:
                edges.append((vid(t, i), vid(t + 1, i)))
            if lattice == TRIANGULAR and t + 1 < N and i >= 1:
                edges.append((vid(t, i), vid(t + 1, i - 1)))
    edges = sorted((min(u, v), max(u, v)) for u, v in edges)
    return L * N, edges


def count_triangles(n, edges):
    """Number of 3-cycles, by brute force over vertex triples."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    c = 0
    for a in range(n):
        for b in adj[a]:
            if b <= a:
                continue
            for d in adj[a] & adj[b]:
                if d > b:
                    c += 1
    return c

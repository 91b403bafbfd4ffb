"""Small hand-made graphs and independent brute-force counters for the tests.

The brute-force routines here are deliberately different algorithms from the
oracle's (subset enumeration, id-ordered bitmask extension) so that they pin
it rather than restate it.
"""
import itertools
import math
import os

import numpy as np

import kclgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_edge_fixture(name):
    n = None
    edges = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "n":
                n = int(parts[1])
            else:
                edges.append((int(parts[0]), int(parts[1])))
    rp, col = kclgen.from_edges(n, edges)
    return rp, col


def csr_from_edges(n, edges):
    return kclgen.from_edges(n, list(edges) if edges else np.zeros((0, 2), np.uint32))


def adjacency_sets(rp, col):
    n = len(rp) - 1
    return [set(int(x) for x in col[rp[u]:rp[u + 1]]) for u in range(n)]


def brute_cliques_subsets(rp, col, k):
    """Every k-subset checked pair by pair (use for small n)."""
    adj = adjacency_sets(rp, col)
    n = len(adj)
    out = []
    for S in itertools.combinations(range(n), k):
        if all(b in adj[a] for a, b in itertools.combinations(S, 2)):
            out.append(S)
    return out


def brute_cliques_bitmask(rp, col, k):
    """Cliques grown in increasing id order with Python-int neighbour masks
    (an explicit-stack search; no degree ordering, no merge joins)."""
    adj = adjacency_sets(rp, col)
    n = len(adj)
    mask = [sum(1 << v for v in adj[u]) for u in range(n)]
    out = []
    for u in range(n):
        if k == 1:
            out.append((u,))
            continue
        stack = [([u], mask[u] & ~((1 << (u + 1)) - 1))]
        while stack:
            R, c = stack.pop()
            if len(R) == k:
                out.append(tuple(R))
                continue
            x = c
            while x:
                low = x & -x
                v = low.bit_length() - 1
                x ^= low
                stack.append((R + [v], c & mask[v] & ~((1 << (v + 1)) - 1)))
    return sorted(out)


def gnp(n, p, seed):
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
    return csr_from_edges(n, edges)


def complete(n):
    return csr_from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)])


def turan(parts):
    """Complete multipartite graph with the given part sizes."""
    lab = []
    for i, s in enumerate(parts):
        lab += [i] * s
    n = len(lab)
    return csr_from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)
                              if lab[u] != lab[v]])


def elementary_symmetric(xs, k):
    e = [1] + [0] * k
    for x in xs:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * x
    return e[k]


def disjoint_union(g1, g2):
    rp1, c1 = g1
    rp2, c2 = g2
    n1 = len(rp1) - 1
    n2 = len(rp2) - 1
    e = []
    for u in range(n1):
        e += [(u, int(v)) for v in c1[rp1[u]:rp1[u + 1]] if u < v]
    for u in range(n2):
        e += [(u + n1, int(v) + n1) for v in c2[rp2[u]:rp2[u + 1]] if u < v]
    return csr_from_edges(n1 + n2, e)


def relabel(g, perm):
    rp, c = g
    n = len(rp) - 1
    e = []
    for u in range(n):
        e += [(int(perm[u]), int(perm[v])) for v in c[rp[u]:rp[u + 1]] if u < v]
    return csr_from_edges(n, e)


def comb(n, k):
    return math.comb(n, k) if 0 <= k <= n else 0


GOLD = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1

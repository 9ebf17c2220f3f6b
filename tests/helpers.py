"""Small graph builders and independent checks shared by the tests.

Nothing here computes the method; these are test inputs and plain checks
(scipy / numpy / networkx library routines, brute force).
"""
import itertools

import numpy as np

from paper_1806_07028_gb300 import inputs as I


def random_graph(n, p, seed, weights="uniform"):
    """Connected Erdos-Renyi-like graph: a random spanning tree plus extra edges."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    ei, ej = [], []
    for k in range(1, n):
        a, b = perm[k], perm[rng.integers(0, k)]
        ei.append(min(a, b)); ej.append(max(a, b))
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                ei.append(a); ej.append(b)
    key = np.unique(np.array(ei, np.int64) * n + np.array(ej, np.int64))
    i, j = key // n, key % n
    w = rng.uniform(0.1, 1.0, i.size) if weights == "uniform" else np.ones(i.size)
    return I.laplacian_from_edges(n, i, j, w, f"er_{n}_{seed}")


def edges_of(rowptr, col, w=None):
    out = {}
    for u in range(len(rowptr) - 1):
        for k in range(rowptr[u], rowptr[u + 1]):
            v = int(col[k])
            if v > u:
                out[(u, v)] = None if w is None else float(w[k])
    return out


def cover_edges(nbr0, nbr1):
    es = set()
    for u in range(len(nbr0)):
        for v in (nbr0[u], nbr1[u]):
            if v >= 0:
                es.add((min(u, int(v)), max(u, int(v))))
    return es


def is_path_cover(n, es):
    """Vertex-disjoint paths: degree <= 2 and no cycle."""
    deg = np.zeros(n, int)
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for (a, b) in es:
        deg[a] += 1; deg[b] += 1
        ra, rb = find(a), find(b)
        if ra == rb:
            return False
        parent[ra] = rb
    return bool(np.all(deg <= 2))


def max_path_cover_weight(n, edges):
    """Brute force over all edge subsets (tiny graphs only)."""
    items = list(edges.items())
    best = 0.0
    for r in range(len(items) + 1):
        for sub in itertools.combinations(items, r):
            es = [e for e, _ in sub]
            if is_path_cover(n, es):
                best = max(best, sum(w for _, w in sub))
    return best


def nbr_lists(nbr0, nbr1):
    return [[int(v) for v in (nbr0[u], nbr1[u]) if v >= 0] for u in range(len(nbr0))]

"""Seeded synthetic inputs: weighted graph Laplacians and right-hand sides.

This module only *creates problem instances* (graphs, their Laplacians, right-hand
sides and test vectors). It holds none of the solver's arithmetic, so both the
CUDA path and the CPU oracle can be fed from it.

A graph Laplacian here is the matrix of Section 2.2 of the paper: for a weighted
undirected graph G = (V, E, w) with w > 0 and no self-loops, A_ij = -w_ij for an
edge (i, j) and A_ii = sum_j w_ij. Storage is CSR with int32 row pointers and
column indices (columns ascending, diagonal stored) and float64 values.

Workload recipes (all seeded, all synthetic):

* ``grid2d``     2D 4-neighbour grid graph, lexicographic order, unit or
                 log-uniform weights 10^U(-3,0) per edge.
* ``grid3d``     3D 7-point grid graph, lexicographic order. Vertex coefficients
                 come from a block pattern (checkerboard 1 / 1e-4 on 8^3 blocks,
                 or log-uniform 10^U(-6,0) per 16^3 block); an edge weighs the
                 harmonic mean of its two endpoint coefficients, x-edges
                 optionally scaled (anisotropy).
* ``ring``       Watts-Strogatz ring lattice with rewiring probability 0
                 (each vertex joined to its k/2 nearest neighbours on each side).
* ``chung_lu``   power-law expected degrees w_i ~ (i + i0)^(-1/(beta-1)), scaled to
                 the requested mean degree; endpoint pairs drawn proportionally to w;
                 self-loops and duplicates dropped; largest connected component
                 kept with vertex order preserved; weights uniform in (0, 1].
* ``rgg``        random geometric graph in the unit square, radius chosen for the
                 requested mean degree, vertices ordered by grid cell then index,
                 largest connected component, weights 1/distance.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Graph", "laplacian_from_edges", "grid2d", "grid3d", "ring", "chung_lu",
    "rgg", "rhs_normal", "rhs_lowfreq", "random_vector", "workload",
    "WORKLOADS",
]


class Graph:
    """A graph Laplacian in CSR form (int32 indices, float64 values)."""

    def __init__(self, rowptr, col, val, name=""):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = int(self.rowptr.shape[0] - 1)
        self.nnz = int(self.col.shape[0])
        self.name = name

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def __repr__(self):
        return f"Graph({self.name!r}, n={self.n}, nnz={self.nnz})"


def laplacian_from_edges(n, i, j, w, name=""):
    """CSR Laplacian of the undirected graph with edges (i[k], j[k], w[k]).

    Each undirected edge must appear once with i != j. Columns come out sorted,
    the diagonal is stored, off-diagonals are -w.
    """
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    if np.any(i == j):
        raise ValueError("self-loops are not allowed")
    if np.any(w <= 0):
        raise ValueError("weights must be positive")
    rows = np.concatenate([i, j, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([j, i, np.arange(n, dtype=np.int64)])
    deg = np.bincount(i, weights=w, minlength=n) + np.bincount(j, weights=w, minlength=n)
    vals = np.concatenate([-w, -w, deg])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if np.any(dup):
            raise ValueError("parallel edges are not allowed")
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return Graph(rowptr.astype(np.int32), cols.astype(np.int32), vals, name)


def grid2d(nx, ny, weights="unit", seed=0):
    """2D grid graph, 4-neighbour edges, vertex id = x + nx*y."""
    rng = np.random.default_rng(seed)
    idx = np.arange(nx * ny).reshape(ny, nx)
    ei = [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
    ej = [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    i = np.concatenate(ei)
    j = np.concatenate(ej)
    if weights == "unit":
        w = np.ones(i.size)
    elif weights == "loguniform":
        w = 10.0 ** rng.uniform(-3.0, 0.0, size=i.size)
    else:
        raise ValueError(weights)
    return laplacian_from_edges(nx * ny, i, j, w, f"grid2d_{nx}x{ny}_{weights}")


def grid3d(nx, ny, nz, coeff="unit", block=8, xscale=1.0, seed=0):
    """3D 7-point grid graph, vertex id = x + nx*(y + ny*z).

    coeff = "unit":         all vertex coefficients 1
    coeff = "checkerboard": coefficient 1 where floor(x/b)+floor(y/b)+floor(z/b)
                            is even, else 1e-4 (b = block)
    coeff = "jumps":        coefficient 10^U(-6,0) drawn per b^3 block
    Edge weight = harmonic mean of its endpoints' coefficients; x-edges are
    multiplied by ``xscale``.
    """
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if coeff == "unit":
        c = np.ones((nz, ny, nx))
    elif coeff == "checkerboard":
        par = (x // block + y // block + z // block) % 2
        c = np.where(par == 0, 1.0, 1e-4)
    elif coeff == "jumps":
        bz, by, bx = -(-nz // block), -(-ny // block), -(-nx // block)
        bc = 10.0 ** rng.uniform(-6.0, 0.0, size=(bz, by, bx))
        c = bc[z // block, y // block, x // block]
    else:
        raise ValueError(coeff)
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)

    def hm(a, b):
        return 2.0 * a * b / (a + b)

    parts_i, parts_j, parts_w = [], [], []
    parts_i.append(idx[:, :, :-1].ravel()); parts_j.append(idx[:, :, 1:].ravel())
    parts_w.append(xscale * hm(c[:, :, :-1], c[:, :, 1:]).ravel())
    parts_i.append(idx[:, :-1, :].ravel()); parts_j.append(idx[:, 1:, :].ravel())
    parts_w.append(hm(c[:, :-1, :], c[:, 1:, :]).ravel())
    parts_i.append(idx[:-1, :, :].ravel()); parts_j.append(idx[1:, :, :].ravel())
    parts_w.append(hm(c[:-1, :, :], c[1:, :, :]).ravel())
    return laplacian_from_edges(nx * ny * nz, np.concatenate(parts_i),
                                np.concatenate(parts_j), np.concatenate(parts_w),
                                f"grid3d_{nx}x{ny}x{nz}_{coeff}")


def ring(n, k=4):
    """Watts-Strogatz lattice with beta = 0: vertex i joined to i+1..i+k/2 (mod n)."""
    i, j = [], []
    for s in range(1, k // 2 + 1):
        a = np.arange(n)
        b = (a + s) % n
        i.append(np.minimum(a, b)); j.append(np.maximum(a, b))
    i = np.concatenate(i); j = np.concatenate(j)
    key = np.unique(i.astype(np.int64) * n + j)
    i, j = key // n, key % n
    return laplacian_from_edges(n, i, j, np.ones(i.size), f"ring_{n}_k{k}")


def _largest_component(n, i, j):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    g = sp.coo_matrix((np.ones(i.size), (i, j)), shape=(n, n))
    ncomp, lab = connected_components(g, directed=False)
    if ncomp == 1:
        return np.arange(n), n
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    return keep, keep.size


def _relabel(n, keep, i, j, w):
    newid = np.full(n, -1, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    m = (newid[i] >= 0) & (newid[j] >= 0)
    return newid[i[m]], newid[j[m]], w[m]


def chung_lu(n, beta=2.1, mean_deg=10.0, seed=0, i0=None):
    """Chung-Lu power-law graph (largest connected component)."""
    rng = np.random.default_rng(seed)
    if i0 is None:
        i0 = max(1.0, n ** 0.1)
    wexp = (np.arange(n) + i0) ** (-1.0 / (beta - 1.0))
    p = wexp / wexp.sum()
    m = int(round(n * mean_deg / 2.0))
    a = rng.choice(n, size=m, p=p)
    b = rng.choice(n, size=m, p=p)
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo.astype(np.int64) * n + hi)
    i, j = key // n, key % n
    w = 1.0 - rng.random(i.size)  # uniform in (0, 1]
    kept, nl = _largest_component(n, i, j)
    i, j, w = _relabel(n, kept, i, j, w)
    return laplacian_from_edges(nl, i, j, w, f"chunglu_{n}_b{beta}")


def rgg(n, mean_deg=12.0, seed=0):
    """Random geometric graph in [0,1]^2 with weights 1/distance (largest component)."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(mean_deg / (np.pi * n))
    pts = rng.random((n, 2))
    ncell = max(1, int(np.floor(1.0 / r)))
    cx = np.minimum((pts[:, 0] * ncell).astype(np.int64), ncell - 1)
    cy = np.minimum((pts[:, 1] * ncell).astype(np.int64), ncell - 1)
    cell = cy * ncell + cx
    order = np.lexsort((np.arange(n), cell))
    pts, cx, cy, cell = pts[order], cx[order], cy[order], cell[order]
    start = np.searchsorted(cell, np.arange(ncell * ncell + 1))
    ii, jj, ww = [], [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ncx, ncy = cx + dx, cy + dy
            ok = (ncx >= 0) & (ncx < ncell) & (ncy >= 0) & (ncy < ncell)
            src = np.flatnonzero(ok)
            nc = ncy[src] * ncell + ncx[src]
            cnt = start[nc + 1] - start[nc]
            rep = np.repeat(src, cnt)
            off = np.repeat(start[nc], cnt) + (np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt))
            m = rep < off
            a, b = rep[m], off[m]
            d = np.sqrt(((pts[a] - pts[b]) ** 2).sum(axis=1))
            m2 = (d <= r) & (d > 0)
            ii.append(a[m2]); jj.append(b[m2]); ww.append(1.0 / d[m2])
    i = np.concatenate(ii); j = np.concatenate(jj); w = np.concatenate(ww)
    kept, nl = _largest_component(n, i, j)
    i, j, w = _relabel(n, kept, i, j, w)
    return laplacian_from_edges(nl, i, j, w, f"rgg_{n}_d{mean_deg}")


def rhs_normal(n, seed=0):
    """Standard normal right-hand side with its mean removed (orthogonal to 1)."""
    b = np.random.default_rng(seed).standard_normal(n)
    return b - b.mean()


def rhs_lowfreq(n):
    """The low-frequency right-hand side [1, ..., 1, 1-n] used in Section 4."""
    b = np.ones(n)
    b[-1] = 1.0 - n
    return b


def random_vector(n, seed=0, kind="normal"):
    """A seeded test vector (e.g. a stand-in smooth error fed to both sides)."""
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal(n)
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, n)
    raise ValueError(kind)


# Named workloads. "C*" follow the five synthetic configurations of the
# performance study; "*-small" are scaled-down copies of the same recipe.
def workload(name, seed=None):
    s = 0 if seed is None else seed
    if name == "C1":
        return grid2d(64, 64, "loguniform", seed=1000 + s)
    if name == "C2":
        return grid3d(128, 128, 128, "checkerboard", block=8, xscale=100.0, seed=2000 + s)
    if name == "C2-small":
        return grid3d(32, 32, 32, "checkerboard", block=8, xscale=100.0, seed=2000 + s)
    if name == "C2-mid":
        return grid3d(64, 64, 64, "checkerboard", block=8, xscale=100.0, seed=2000 + s)
    if name == "C3":
        return chung_lu(1_000_000, 2.1, 10.0, seed=3000 + s)
    if name == "C3-small":
        return chung_lu(20_000, 2.1, 10.0, seed=3000 + s)
    if name == "C4":
        return rgg(2_000_000, 12.0, seed=4000 + s)
    if name == "C4-small":
        return rgg(20_000, 12.0, seed=4000 + s)
    if name == "C5":
        return grid3d(256, 256, 256, "jumps", block=16, xscale=1.0, seed=5000 + s)
    if name == "C5-small":
        return grid3d(32, 32, 32, "jumps", block=16, xscale=1.0, seed=5000 + s)
    if name == "C5-mid":
        return grid3d(128, 128, 128, "jumps", block=16, xscale=1.0, seed=5000 + s)
    if name.startswith("grid2d-unit-"):
        k = int(name.rsplit("-", 1)[1])
        return grid2d(k, k, "unit")
    if name.startswith("ring-"):
        return ring(int(name.rsplit("-", 1)[1]), 4)
    raise KeyError(name)


WORKLOADS = ["C1", "C2", "C2-small", "C2-mid", "C3", "C3-small", "C4", "C4-small",
             "C5", "C5-small", "C5-mid"]

# One-line statement of each workload's recipe and size, for reports.
DESCRIPTIONS = {
    "C1": "2D 4-neighbour grid Laplacian 64x64 (n = 4,096), edge weights 10^U(-3,0)",
    "C2": "3D 7-point grid Laplacian 128^3 (n = 2,097,152), 8^3 checkerboard weights 1 / 1e-4, "
          "x-edges x100",
    "C2-small": "3D 7-point grid 32^3, C2's checkerboard weights and anisotropy",
    "C2-mid": "3D 7-point grid 64^3, C2's checkerboard weights and anisotropy",
    "C3": "Chung-Lu scale-free graph, exponent 2.1, n = 1,000,000, mean degree 10, largest component, "
          "weights U(0,1]",
    "C3-small": "Chung-Lu scale-free graph, exponent 2.1, n = 20,000, largest component",
    "C4": "random geometric graph in the unit square, n = 2,000,000, mean degree 12, largest component, "
          "weights 1/distance",
    "C4-small": "random geometric graph, n = 20,000, mean degree 12",
    "C5": "3D 7-point grid Laplacian 256^3 (n = 16,777,216), jump coefficients 10^U(-6,0) on 16^3 blocks",
    "C5-small": "3D 7-point grid 32^3, C5's block jump coefficients",
    "C5-mid": "3D 7-point grid 128^3 (n = 2,097,152), C5's block jump coefficients on 16^3 blocks",
}


def mpnn_init_params(seed=0):
    """Seeded initial weights of the learned start-vector network, FP32: every
    weight matrix uniform in +-1/sqrt(fan_in), biases zero, in the flat order
    W_in (64x3), b_in (64), [W_l (64x128), b_l (64)] x 4, w_out (64), b_out (1)."""
    rng = np.random.default_rng(seed)
    shapes = [((64, 3), 3), ((64,), 0)] + [((64, 128), 128), ((64,), 0)] * 4 + [((64,), 64), ((1,), 0)]
    parts = []
    for shape, fan_in in shapes:
        if fan_in == 0:
            parts.append(np.zeros(shape).ravel())
        else:
            a = 1.0 / np.sqrt(fan_in)
            parts.append(rng.uniform(-a, a, shape).ravel())
    return np.concatenate(parts).astype(np.float32)

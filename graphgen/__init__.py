"""Seeded synthetic graph generators shared by the oracle tests, the CUDA-path
tests and the benchmark.

This module holds no arithmetic of the partitioning method: it only builds
inputs.  Every graph is returned in canonical undirected CSR form:

* ``row_ptr``: int64[n+1], ``col``: int32[row_ptr[n]];
* symmetric (every arc (u,v) has its twin (v,u)), no self-loops,
  duplicates merged, each row sorted by neighbour id;
* unit int32 weights unless a weight generator below is used.

The paper's instances (web graphs, social networks; its Table 1) are not
available, so R-MAT stands in for the scale-free complex networks and 2D
random geometric graphs stand in for the mesh-like contrast case.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph", "from_edges", "rmat", "rgg2d", "path", "grid", "clique_ring",
    "gnp", "star", "random_weights", "batch_workload", "validate",
]


@dataclass
class Graph:
    """Canonical undirected CSR graph with int32 node and edge weights."""
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [m2]  (m2 = 2 * undirected edges)
    node_w: np.ndarray           # int32 [n]
    edge_w: np.ndarray           # int32 [m2]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def arcs(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def edges(self) -> int:
        return self.arcs // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def from_edges(n: int, src, dst, name: str = "", w=None) -> Graph:
    """Build the canonical CSR from an undirected edge list.

    Self-loops are dropped, both directions are inserted, duplicate arcs are
    merged.  With ``w`` given, duplicates keep the weight of the first
    occurrence of the undirected pair (weights are per undirected edge, so
    both arcs of an edge carry the same weight).
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    key = lo * n + hi
    if w is None:
        key = np.unique(key)
        wu = np.ones(key.shape[0], dtype=np.int32)
    else:
        w = np.asarray(w, dtype=np.int64)[keep]
        key, first = np.unique(key, return_index=True)
        wu = w[first].astype(np.int32)
    lo = key // n
    hi = key % n
    a = np.concatenate([lo, hi])
    b = np.concatenate([hi, lo])
    ww = np.concatenate([wu, wu])
    order = np.lexsort((b, a))
    a, b, ww = a[order], b[order], ww[order]
    counts = np.bincount(a, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(row_ptr, b.astype(np.int32), np.ones(n, dtype=np.int32),
                 ww.astype(np.int32), name=name)


def validate(g: Graph) -> None:
    """Raise ValueError unless ``g`` is canonical (used by tests)."""
    n = g.n
    rp, col = g.row_ptr, g.col
    if rp[0] != 0 or np.any(np.diff(rp) < 0):
        raise ValueError("row_ptr not monotone")
    if col.size and (col.min() < 0 or col.max() >= n):
        raise ValueError("col out of range")
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    if np.any(src == col):
        raise ValueError("self-loop")
    k1 = src * n + col
    if np.unique(k1).size != k1.size:
        raise ValueError("duplicate arc")
    k2 = col.astype(np.int64) * n + src
    o1, o2 = np.argsort(k1), np.argsort(k2)
    if not np.array_equal(k1[o1], k2[o2]):
        raise ValueError("not symmetric")
    if not np.array_equal(g.edge_w[o1], g.edge_w[o2]):
        raise ValueError("asymmetric edge weights")
    if np.any(g.edge_w <= 0) or np.any(g.node_w <= 0):
        raise ValueError("weights must be positive")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
         permute: bool = True) -> Graph:
    """R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004).

    ``edge_factor * 2**scale`` edges are sampled; each picks one quadrant of
    the adjacency matrix per bit with probabilities (a, b, c, d=1-a-b-c).
    Self-loops are dropped, duplicates merged, the graph symmetrised, and
    node ids permuted at random so that hubs are not packed at low ids.
    """
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(np.random.SeedSequence([0x524D4154, scale, edge_factor, seed]))
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    chunk = 1 << 22
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        sv = np.zeros(e - s, dtype=np.int64)
        dv = np.zeros(e - s, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(e - s)
            sbit = (r >= ab).astype(np.int64)
            dbit = (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64)
            sv = (sv << 1) | sbit
            dv = (dv << 1) | dbit
        src[s:e] = sv
        dst[s:e] = dv
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        src, dst = perm[src], perm[dst]
    g = from_edges(n, src, dst, name=f"rmat-s{scale}-ef{edge_factor}-seed{seed}")
    g.meta.update(kind="rmat", scale=scale, edge_factor=edge_factor, seed=seed)
    return g


def rgg2d(n: int, seed: int, radius_factor: float = 0.55) -> Graph:
    """2D random geometric graph: ``n`` points uniform in the unit square,
    an edge between every pair closer than r = radius_factor*sqrt(ln n / n)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(np.random.SeedSequence([0x524747, n, seed]))
    pts = rng.random((n, 2))
    r = radius_factor * math.sqrt(math.log(n) / n)
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    g = from_edges(n, pairs[:, 0], pairs[:, 1], name=f"rgg2d-n{n}-seed{seed}")
    g.meta.update(kind="rgg", n=n, seed=seed, radius=r)
    return g


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"path-{n}")


def grid(rows: int, cols: int) -> Graph:
    idx = np.arange(rows * cols).reshape(rows, cols)
    s = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    d = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(rows * cols, s, d, name=f"grid-{rows}x{cols}")


def clique_ring(k: int, s: int, ring: bool = True) -> Graph:
    """``k`` cliques of ``s`` nodes; clique i's last node is joined to clique
    i+1's first node (cyclically when ``ring``, else as a path of cliques)."""
    src, dst = [], []
    for q in range(k):
        base = q * s
        a, b = np.triu_indices(s, 1)
        src.append(base + a)
        dst.append(base + b)
    links = k if ring else k - 1
    for q in range(links):
        src.append(np.array([q * s + s - 1]))
        dst.append(np.array([((q + 1) % k) * s]))
    return from_edges(k * s, np.concatenate(src), np.concatenate(dst),
                      name=f"cliques-{k}x{s}{'-ring' if ring else '-path'}")


def star(leaves: int) -> Graph:
    return from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64),
                      np.arange(1, leaves + 1), name=f"star-{leaves}")


def gnp(n: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(np.random.SeedSequence([0x474E50, n, seed]))
    a, b = np.triu_indices(n, 1)
    keep = rng.random(a.size) < p
    return from_edges(n, a[keep], b[keep], name=f"gnp-{n}-{p}-{seed}")


def random_weights(g: Graph, seed: int, max_node_w: int = 4, max_edge_w: int = 8) -> Graph:
    """Same graph with random positive weights (symmetric per edge)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x575453, g.n, g.arcs, seed]))
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    lo = np.minimum(src, g.col)
    hi = np.maximum(src, g.col)
    key = lo * n + hi
    uk, inv = np.unique(key, return_inverse=True)
    wu = rng.integers(1, max_edge_w + 1, size=uk.size).astype(np.int32)
    nw = rng.integers(1, max_node_w + 1, size=n).astype(np.int32)
    return Graph(g.row_ptr.copy(), g.col.copy(), nw, wu[inv].astype(np.int32),
                 name=g.name + f"-w{seed}", meta=dict(g.meta))


def batch_params(i: int, count: int = 512, seed: int = 0):
    """Parameters of graph ``i`` of the batched workload: even i -> R-MAT with
    scale uniform in 10..16 (edge factor 8), odd i -> 2D RGG with n
    log-uniform in 1k..64k; k uniform in {2,4,8,16}; eps = 0.03."""
    rng = np.random.default_rng(np.random.SeedSequence([0x42415443, count, seed, i]))
    k = int(rng.choice([2, 4, 8, 16]))
    if i % 2 == 0:
        return dict(kind="rmat", scale=int(rng.integers(10, 17)), k=k, eps=0.03,
                    gseed=1000 * seed + i)
    n = int(round(math.exp(rng.uniform(math.log(1000), math.log(65536)))))
    return dict(kind="rgg", n=n, k=k, eps=0.03, gseed=1000 * seed + i)


def batch_graph(i: int, count: int = 512, seed: int = 0):
    """Graph ``i`` of the batched workload as (Graph, k, eps)."""
    p = batch_params(i, count, seed)
    if p["kind"] == "rmat":
        g = rmat(p["scale"], 8, seed=p["gseed"])
    else:
        g = rgg2d(p["n"], seed=p["gseed"])
    return g, p["k"], p["eps"]


def batch_workload(count: int = 512, seed: int = 0, processes: int = 0):
    """The batched workload: ``count`` independent graphs of uneven size
    (see batch_params).  Returns a list of (Graph, k, eps).  With
    processes > 1 the graphs are generated by a spawn-started process pool
    (results do not depend on it)."""
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.starmap(batch_graph, [(i, count, seed) for i in range(count)])
    return [batch_graph(i, count, seed) for i in range(count)]

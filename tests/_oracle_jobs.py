"""Oracle jobs run in spawn-started worker processes by the large GPU parity
tests (the oracle is single-threaded; two of these overlap each other and
the GPU work).  Imports no CUDA code."""
import numpy as np

import graphgen as gg
import oracle as O


def partition(row_ptr, col, k, eps, seed):
    """The oracle's partition of a unit-weight graph: (block, cut, status,
    level sizes)."""
    g = gg.Graph(row_ptr, col, np.ones(row_ptr.size - 1, np.int32), np.ones(col.size, np.int32))
    r = O.partition(g, k, eps, seed=seed, unit=True)
    return r.block, r.cut, r.status, list(r.stats.level_n[:r.stats.levels])


def rgg_and_partition(n, gseed, k, eps, seed):
    """Generates the 2D RGG on the host and partitions it with the oracle:
    (row_ptr, col, block, cut, status, level sizes)."""
    g = gg.rgg2d(n, gseed)
    r = O.partition(g, k, eps, seed=seed)
    return g.row_ptr, g.col, r.block, r.cut, r.status, list(r.stats.level_n[:r.stats.levels])

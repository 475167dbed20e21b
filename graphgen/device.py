"""R-MAT graphs generated where they will be used (torch tensors on any
device), for inputs too large to build with NumPy on the host.

Same model as ``graphgen.rmat`` (Chakrabarti, Zhan, Faloutsos 2004): each of
``edge_factor * 2**scale`` edges picks one quadrant of the adjacency matrix
per bit with probabilities (a, b, c, d = 1 - a - b - c); self-loops are
dropped, duplicates merged, the graph symmetrised, node ids permuted, rows
sorted by neighbour id.  The random draws are not NumPy's: draw (e, l) (edge
e, bit l) is the SplitMix64 output (Steele, Lea, Flood, OOPSLA 2014) at
counter 64 e + l of a stream keyed by (scale, edge_factor, seed), compared as
a 53-bit integer against the quadrant thresholds, so the graph is the same
on every device and for every chunk and part size (it differs from
``graphgen.rmat`` for the same seed).

Like the rest of ``graphgen`` this module builds inputs only and holds none
of the partitioning method's arithmetic.
"""
from __future__ import annotations

import math

__all__ = ["rmat_torch", "splitmix64_py"]

_M64 = (1 << 64) - 1
_GOLD = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """Python int (mod 2^64) as the int64 value with the same bits."""
    x &= _M64
    return x - (1 << 64) if x >> 63 else x


def splitmix64_py(z: int) -> int:
    """SplitMix64 output function on a Python int, exact mod 2^64."""
    z &= _M64
    z = ((z ^ (z >> 30)) * _C1) & _M64
    z = ((z ^ (z >> 27)) * _C2) & _M64
    return z ^ (z >> 31)


def _srl(z, k: int):
    """Logical right shift of an int64 tensor (>> is arithmetic on int64)."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _splitmix64_t(z):
    """SplitMix64 output function on an int64 tensor (products wrap mod 2^64)."""
    z = (z ^ _srl(z, 30)) * _s64(_C1)
    z = (z ^ _srl(z, 27)) * _s64(_C2)
    return z ^ _srl(z, 31)


def _permute(x, scale: int, key: int):
    """A keyed bijection of [0, 2^scale): three rounds of add, multiply by an
    odd constant and xorshift, each a bijection modulo 2^scale."""
    mask = (1 << scale) - 1
    shift = scale // 2 + 1
    for r in range(3):
        k = splitmix64_py(key + r)
        x = (x + (k & mask)) & mask
        x = (x * (((k >> 32) | 1) & mask | 1)) & mask
        x = x ^ (x >> shift)
    return x


def rmat_torch(scale: int, edge_factor: int, seed: int, device="cpu", a=0.57, b=0.19,
               c=0.19, edge_chunk: int = 1 << 24, parts: int = 0):
    """R-MAT graph as (row_ptr int64[n+1], col int32[arcs]) tensors on ``device``.

    ``edge_chunk`` edges are sampled per pass and ``parts`` node ranges are
    de-duplicated one at a time (0: one part per 2^28 sampled edges); neither
    changes the result, only the temporary memory.
    """
    import torch

    if not 1 <= scale <= 30:
        raise ValueError("scale must be in [1, 30]")
    dev = torch.device(device)
    n = 1 << scale
    m = edge_factor * n
    t_a, t_ab, t_abc = (int(math.floor(p * (1 << 53))) for p in (a, a + b, a + b + c))
    skey = splitmix64_py((0x524D4154 << 32) ^ (scale << 24) ^ (edge_factor << 8) ^ seed)
    pkey = splitmix64_py(skey ^ 0x5045524D)

    lo_parts, hi_parts = [], []
    for s in range(0, m, edge_chunk):
        e = min(m, s + edge_chunk)
        ctr = torch.arange(s, e, device=dev, dtype=torch.int64) * 64
        sv = torch.zeros(e - s, dtype=torch.int64, device=dev)
        dv = torch.zeros(e - s, dtype=torch.int64, device=dev)
        for lvl in range(scale):
            u = _srl(_splitmix64_t(_s64(skey) + (ctr + lvl) * _s64(_GOLD)), 11)
            sbit = u >= t_ab
            dbit = ((u >= t_a) & (u < t_ab)) | (u >= t_abc)
            sv = (sv << 1) | sbit.to(torch.int64)
            dv = (dv << 1) | dbit.to(torch.int64)
        sv = _permute(sv, scale, pkey)
        dv = _permute(dv, scale, pkey)
        keep = sv != dv
        lo_parts.append(torch.minimum(sv, dv)[keep].to(torch.int32))
        hi_parts.append(torch.maximum(sv, dv)[keep].to(torch.int32))
    lo = torch.cat(lo_parts)
    hi = torch.cat(hi_parts)
    del lo_parts, hi_parts

    # undirected edges, de-duplicated by ranges of the smaller endpoint
    P = parts if parts > 0 else max(1, -(-m // (1 << 28)))
    R = -(-n // P)
    ukeys = []
    for p in range(P):
        sel = (lo >= p * R) & (lo < (p + 1) * R)
        ukeys.append(torch.unique(lo[sel].to(torch.int64) * n + hi[sel].to(torch.int64)))
    del lo, hi

    deg = torch.zeros(n, dtype=torch.int64, device=dev)
    for k in ukeys:
        deg += torch.bincount(k // n, minlength=n) + torch.bincount(k % n, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(deg, 0)
    col = torch.empty(int(row_ptr[-1]), dtype=torch.int32, device=dev)

    # row v: first its smaller neighbours (arcs v -> lo of keys (lo, v)), in
    # increasing lo, then its larger ones (keys (v, hi)), in increasing hi;
    # parts are visited in increasing lo and keys are sorted within a part
    placed = torch.zeros(n, dtype=torch.int64, device=dev)
    for k in ukeys:
        h = k % n
        hs, order = torch.sort(h, stable=True)
        ls = (k // n)[order]
        cnt = torch.bincount(hs, minlength=n)
        start = torch.cumsum(cnt, 0) - cnt
        rank = torch.arange(hs.numel(), device=dev, dtype=torch.int64) - start[hs]
        col[row_ptr[hs] + placed[hs] + rank] = ls.to(torch.int32)
        placed += cnt
    for k in ukeys:
        lk = k // n
        cnt = torch.bincount(lk, minlength=n)
        start = torch.cumsum(cnt, 0) - cnt
        rank = torch.arange(lk.numel(), device=dev, dtype=torch.int64) - start[lk]
        col[row_ptr[lk] + placed[lk] + rank] = (k % n).to(torch.int32)
    return row_ptr, col

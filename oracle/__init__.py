"""ctypes wrapper around the CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The product path never imports it.
Builds the library on first use if it is missing (plain g++, no CUDA).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "sclap_oracle.cpp")]

SYNC, SEQ = 0, 1
MODE_CLUSTER, MODE_REFINE = 0, 1
PH_CLUSTER, PH_REFINE, PH_TRIAL, PH_GGG, PH_IPREF, PH_REPAIR, PH_ENSEMBLE, PH_VCYCLE = (
    1, 2, 3, 4, 5, 6, 7, 8)
OK, EINVAL, EOVERFLOW, EINFEASIBLE = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (portable flags, no -march)."""
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "sclap_oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp] + _SRC)
        os.replace(tmp, _SO)
    return _SO


class Config(C.Structure):
    _fields_ = [(name, C.c_int32) for name in (
        "lp_rounds_coarse", "lp_rounds_refine", "f", "coarse_min_nodes",
        "ip_trials", "sub_rounds", "repair_rounds", "max_levels", "cluster_active",
        "random_order", "ensemble", "ensemble_size", "vcycles")]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("level_n", C.c_int64 * 64),
                ("level_m", C.c_int64 * 64), ("cluster_rounds", C.c_int32 * 64),
                ("refine_rounds", C.c_int32 * 64), ("ip_best_trial", C.c_int32),
                ("ip_cut", C.c_int64), ("Lmax", C.c_int64), ("U", C.c_int64),
                ("repair_rounds", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        p = C.c_void_p
        i32, i64, u64, dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "orc_default_config": (None, [p]),
            "orc_mix64": (u64, [u64]),
            "orc_hkey": (u64, [u64, u64, u64, u64]),
            "orc_bounds": (C.c_int, [i64, i32, i32, dbl, i32, p, p]),
            "orc_lp_round": (C.c_int, [i32, i64, p, p, p, p, p, p, i64, i64, u64, i32, p, p, p]),
            "orc_cluster": (C.c_int, [i32, i64, p, p, p, p, i64, u64, i32, p, p, p]),
            "orc_contract": (C.c_int, [i64, p, p, p, p, p, p, p, p, p, p, p, p]),
            "orc_cluster_hierarchy": (C.c_int, [i32, i64, p, p, p, p, i64, i64, u64, p, p, p,
                                                p, i32]),
            "orc_overlay": (C.c_int, [i64, p, p, p]),
            "orc_cluster_in_blocks": (C.c_int, [i32, i64, p, p, p, p, i64, u64, i32, p, p, p,
                                                p]),
            "orc_ggg": (C.c_int, [i64, p, p, p, p, i32, i64, u64, i32, p, p]),
            "orc_initial_partition": (C.c_int, [i32, i64, p, p, p, p, i32, i64, i64, u64, i32,
                                                p, p, p, p]),
            "orc_refine": (C.c_int, [i32, i64, p, p, p, p, i32, i64, u64, i32, i32, p, p, p]),
            "orc_repair": (C.c_int, [i64, p, p, p, p, i32, i64, u64, p, p, p]),
            "orc_cut": (i64, [i64, p, p, p, p]),
            "orc_partition": (C.c_int, [i32, i64, p, p, p, p, i32, dbl, u64, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def config(**kw) -> Config:
    c = Config()
    lib().orc_default_config(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, int(v))
    return c


def _graph_arrays(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    nw = np.ascontiguousarray(g.node_w, dtype=np.int32)
    ew = np.ascontiguousarray(g.edge_w, dtype=np.int32)
    return rp, col, nw, ew


def mix64(x: int) -> int:
    return int(lib().orc_mix64(x & (2**64 - 1)))


def hkey(seed: int, phase: int, level: int, rnd: int) -> int:
    m = 2**64 - 1
    return int(lib().orc_hkey(seed & m, phase & m, level & m, rnd & m))


def bounds(cV: int, max_c: int, k: int, eps: float, f: int = 18):
    L, U = C.c_int64(), C.c_int64()
    rc = lib().orc_bounds(cV, max_c, k, eps, f, C.byref(L), C.byref(U))
    if rc:
        raise ValueError(f"orc_bounds rc={rc}")
    return L.value, U.value


def lp_round(g, mode, label, W, bound, rkey, sub_rounds, active_cur=None, want_next=False):
    """One synchronous LP round; returns (label, W, moved, active_next)."""
    rp, col, nw, ew = _graph_arrays(g)
    label = np.array(label, dtype=np.int32, copy=True)
    W = np.array(W, dtype=np.int64, copy=True)
    ac = None if active_cur is None else np.ascontiguousarray(active_cur, dtype=np.uint8)
    an = np.zeros(g.n, dtype=np.uint8) if want_next else None
    moved = C.c_int64()
    rc = lib().orc_lp_round(mode, g.n, _p(rp), _p(col), _p(nw), _p(ew), _p(label), _p(W),
                            W.size, bound, rkey & (2**64 - 1), sub_rounds, _p(ac), _p(an),
                            C.byref(moved))
    if rc:
        raise RuntimeError(f"orc_lp_round rc={rc}")
    return label, W, moved.value, an


def cluster(g, U, seed, level=0, variant=SYNC, cfg=None):
    rp, col, nw, ew = _graph_arrays(g)
    label = np.empty(g.n, dtype=np.int32)
    rounds = C.c_int32()
    cfg = cfg or config()
    rc = lib().orc_cluster(variant, g.n, _p(rp), _p(col), _p(nw), _p(ew), U, seed, level,
                           C.byref(cfg), _p(label), C.byref(rounds))
    if rc:
        raise RuntimeError(f"orc_cluster rc={rc}")
    return label, rounds.value


def cluster_in_blocks(g, U, seed, blk, level=0, variant=SYNC, cfg=None):
    """Clustering in which every cluster lies inside one block of blk."""
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.ascontiguousarray(blk, dtype=np.int32)
    label = np.empty(g.n, dtype=np.int32)
    rounds = C.c_int32()
    cfg = cfg or config()
    rc = lib().orc_cluster_in_blocks(variant, g.n, _p(rp), _p(col), _p(nw), _p(ew), U, seed,
                                     level, C.byref(cfg), _p(blk), _p(label), C.byref(rounds))
    if rc:
        raise RuntimeError(f"orc_cluster_in_blocks rc={rc}")
    return label, rounds.value


def overlay(a, b):
    """Overlay of two clusterings, ids numbered by first occurrence."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    out = np.empty(a.size, dtype=np.int32)
    rc = lib().orc_overlay(a.size, _p(a), _p(b), _p(out))
    if rc:
        raise RuntimeError(f"orc_overlay rc={rc}")
    return out


def cluster_hierarchy(g, U, stop_nodes, seed, variant=SYNC, cfg=None):
    """Clustering hierarchy without k: (community of each input node,
    contractions kept, node counts per level, input first)."""
    rp, col, nw, ew = _graph_arrays(g)
    comm = np.empty(g.n, dtype=np.int32)
    levels = C.c_int32()
    cap = 65
    level_n = np.zeros(cap, dtype=np.int64)
    cfg = cfg or config()
    rc = lib().orc_cluster_hierarchy(variant, g.n, _p(rp), _p(col), _p(nw), _p(ew), int(U),
                                     int(stop_nodes), seed & (2**64 - 1), C.byref(cfg),
                                     _p(comm), C.byref(levels), _p(level_n), cap)
    if rc:
        raise RuntimeError(f"orc_cluster_hierarchy rc={rc}")
    return comm, levels.value, [int(x) for x in level_n[:levels.value + 1]]


@dataclass
class Coarse:
    cmap: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    node_w: np.ndarray
    edge_w: np.ndarray

    @property
    def n(self):
        return int(self.row_ptr.size - 1)


def contract(g, label) -> Coarse:
    rp, col, nw, ew = _graph_arrays(g)
    label = np.ascontiguousarray(label, dtype=np.int32)
    n, m = g.n, g.arcs
    cmap = np.empty(n, np.int32)
    cnw = np.empty(n, np.int32)
    cxadj = np.empty(n + 1, np.int64)
    cadj = np.empty(max(m, 1), np.int32)
    cew = np.empty(max(m, 1), np.int32)
    nc, mc = C.c_int64(), C.c_int64()
    rc = lib().orc_contract(n, _p(rp), _p(col), _p(nw), _p(ew), _p(label), _p(cmap),
                            C.byref(nc), _p(cnw), _p(cxadj), _p(cadj), _p(cew), C.byref(mc))
    if rc:
        raise RuntimeError(f"orc_contract rc={rc}")
    a, b = nc.value, mc.value
    return Coarse(cmap, cxadj[:a + 1].copy(), cadj[:b].copy(), cnw[:a].copy(), cew[:b].copy())


def ggg(g, k, avg, tkey, level=0):
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.empty(g.n, np.int32)
    W = np.empty(k, np.int64)
    lib().orc_ggg(g.n, _p(rp), _p(col), _p(nw), _p(ew), k, avg, tkey & (2**64 - 1), level,
                  _p(blk), _p(W))
    return blk, W


def initial_partition(g, k, Lmax, avg, seed, level=0, variant=SYNC, cfg=None):
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.empty(g.n, np.int32)
    cut, best = C.c_int64(), C.c_int32()
    cfg = cfg or config()
    rc = lib().orc_initial_partition(variant, g.n, _p(rp), _p(col), _p(nw), _p(ew), k, Lmax,
                                     avg, seed, level, C.byref(cfg), _p(blk), C.byref(cut),
                                     C.byref(best))
    if rc:
        raise RuntimeError(f"orc_initial_partition rc={rc}")
    return blk, cut.value, best.value


def refine(g, k, Lmax, block, seed, phase=PH_REFINE, level=0, variant=SYNC, cfg=None):
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.array(block, dtype=np.int32, copy=True)
    rounds = C.c_int32()
    cfg = cfg or config()
    rc = lib().orc_refine(variant, g.n, _p(rp), _p(col), _p(nw), _p(ew), k, Lmax, seed, phase,
                          level, C.byref(cfg), _p(blk), C.byref(rounds))
    if rc:
        raise RuntimeError(f"orc_refine rc={rc}")
    return blk, rounds.value


def repair(g, k, Lmax, block, seed, cfg=None):
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.array(block, dtype=np.int32, copy=True)
    rounds = C.c_int32()
    cfg = cfg or config()
    rc = lib().orc_repair(g.n, _p(rp), _p(col), _p(nw), _p(ew), k, Lmax, seed, C.byref(cfg),
                          _p(blk), C.byref(rounds))
    return blk, rounds.value, rc


def cut(g, block) -> int:
    rp, col, nw, ew = _graph_arrays(g)
    b = np.ascontiguousarray(block, dtype=np.int32)
    return int(lib().orc_cut(g.n, _p(rp), _p(col), _p(ew), _p(b)))


@dataclass
class Result:
    block: np.ndarray
    cut: int
    max_block_weight: int
    status: int
    stats: Stats


def partition(g, k, eps=0.03, seed=0, variant=SYNC, cfg=None, unit=False) -> Result:
    rp, col, nw, ew = _graph_arrays(g)
    blk = np.empty(g.n, np.int32)
    cutv, mb = C.c_int64(), C.c_int64()
    st = Stats()
    cfg = cfg or config()
    rc = lib().orc_partition(variant, g.n, _p(rp), _p(col), None if unit else _p(nw),
                             None if unit else _p(ew), k, eps, seed, C.byref(cfg), _p(blk),
                             C.byref(cutv), C.byref(mb), C.byref(st))
    if rc not in (OK, EINFEASIBLE):
        raise RuntimeError(f"orc_partition rc={rc}")
    return Result(blk, cutv.value, mb.value, rc, st)

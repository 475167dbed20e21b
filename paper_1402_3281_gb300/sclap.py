"""Python binding of the C ABI in include/sclap.h (ctypes).

Argument marshalling only: every step runs in libsclap.so's CUDA kernels.
Host arrays are numpy arrays; device arrays are CUDA torch tensors.  Loading
fails loudly if the library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SCLAP_LIBRARY selects another build of the same ABI (the bounds-check
# build, libsclap_check.so); the default is the in-tree libsclap.so
LIB_PATH = os.environ.get("SCLAP_LIBRARY") or os.path.join(_HERE, "libsclap.so")

OK, EINVAL, ECSR, ENOMEM, ECUDA, EOVERFLOW, EINFEASIBLE, ETIMEOUT, EINTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
PENDING = 1
MODE_CLUSTER, MODE_REFINE = 0, 1
PH_REFINE, PH_IPREF = 2, 5

SYMBOLS = (
    "sclap_default_config", "sclap_error_string", "sclap_last_error", "sclap_partition",
    "sclap_partition_device", "sclap_partition_batch", "sclap_lp_round", "sclap_cluster",
    "sclap_contract", "sclap_cluster_hierarchy", "sclap_initial_partition", "sclap_refine", "sclap_cut",
    "sclap_cut_static", "sclap_server_create", "sclap_server_submit", "sclap_server_poll",
    "sclap_server_destroy", "sclap_get_tuning", "sclap_set_tuning", "sclap_autotune",
    "sclap_profile_enable", "sclap_profile_reset", "sclap_profile_read",
    "sclap_profile_timeline", "sclap_profile_dump", "sclap_profile_phases",
    "sclap_debug_inject", "sclap_check_build", "sclap_check_selftest",
)


class SclapError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib().sclap_error_string(code).decode()
        detail = _lib().sclap_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")
        self.code = code


class Config(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "lp_rounds_coarse", "lp_rounds_refine", "f", "coarse_min_nodes", "ip_trials",
        "sub_rounds", "repair_rounds", "max_levels", "cluster_active", "graph_rounds",
        "ensemble", "ensemble_size", "vcycles")]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("level_n", C.c_int64 * 64), ("level_m", C.c_int64 * 64),
                ("cluster_rounds", C.c_int32 * 64), ("refine_rounds", C.c_int32 * 64),
                ("ip_best_trial", C.c_int32), ("ip_cut", C.c_int64), ("Lmax", C.c_int64),
                ("U", C.c_int64), ("lp_arcs", C.c_int64)]

    def to_dict(self) -> dict:
        L = self.levels
        return dict(levels=L, level_n=list(self.level_n[:L]), level_m=list(self.level_m[:L]),
                    cluster_rounds=list(self.cluster_rounds[:L]),
                    refine_rounds=list(self.refine_rounds[:L]),
                    ip_best_trial=self.ip_best_trial, ip_cut=self.ip_cut, Lmax=self.Lmax,
                    U=self.U, lp_arcs=self.lp_arcs)


class Profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("propose_launches", C.c_int64 * 4),
                ("propose_ms", C.c_double * 4), ("propose_nodes", C.c_int64 * 4),
                ("propose_arcs", C.c_int64 * 4), ("sweep_ms", C.c_double),
                ("sweeps", C.c_int64), ("propose_arcs_unit", C.c_int64)]

    def to_dict(self) -> dict:
        return dict(kernel_launches=self.kernel_launches,
                    propose_launches=list(self.propose_launches),
                    propose_ms=list(self.propose_ms), propose_nodes=list(self.propose_nodes),
                    propose_arcs=list(self.propose_arcs), sweep_ms=self.sweep_ms,
                    sweeps=self.sweeps, propose_arcs_unit=self.propose_arcs_unit)


class ServerOptions(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_int64), ("workers", C.c_int32),
                ("max_batch", C.c_int32), ("linger_us", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("small_max_deg", "small_ctas_per_sm",
                                         "warp_ctas_per_sm", "admit_ctas_per_sm", "concurrent",
                                         "pdl", "fused_admission", "contract_table_slots",
                                         "ip_trial_group", "contract_merge")]

    def to_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class GraphDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("node_w", C.c_void_p), ("edge_w", C.c_void_p), ("k", C.c_int32),
                ("eps", C.c_double), ("seed", C.c_uint64), ("block_out", C.c_void_p),
                ("cut", C.c_int64), ("max_block_weight", C.c_int64), ("status", C.c_int32)]


_handle = None


def _lib():
    global _handle
    if _handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1402_3281_gb300.build` "
                "(the partitioner has no CPU fallback)")
        h = C.CDLL(LIB_PATH)
        p, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "sclap_default_config": (None, [p]),
            "sclap_error_string": (C.c_char_p, [C.c_int]),
            "sclap_last_error": (C.c_char_p, []),
            "sclap_partition": (C.c_int, [i64, p, p, p, p, i32, dbl, u64, p, p, p, p, p]),
            "sclap_partition_device": (C.c_int, [i64, p, p, p, p, i32, dbl, u64, p, p, p, p, p, p]),
            "sclap_partition_batch": (C.c_int, [i32, p, p, i32, p]),
            "sclap_lp_round": (C.c_int, [i32, i64, p, p, p, p, p, p, i64, i64, u64, i32, p, p, p, p]),
            "sclap_cluster": (C.c_int, [i64, p, p, p, p, i64, u64, i32, p, p, p, p]),
            "sclap_contract": (C.c_int, [i64, p, p, p, p, p, p, p, p, p, p, p, p, p]),
            "sclap_cluster_hierarchy": (C.c_int, [i64, p, p, p, p, i64, i64, u64, p, p, p, p,
                                                  i32, p]),
            "sclap_initial_partition": (C.c_int, [i64, p, p, p, p, i32, i64, i64, u64, i32, p, p,
                                                  p, p, p]),
            "sclap_refine": (C.c_int, [i64, p, p, p, p, i32, i64, u64, i32, i32, p, p, p, p]),
            "sclap_cut": (C.c_int, [i64, p, p, p, p, p, p]),
            "sclap_cut_static": (C.c_int, [i64, p, p, p, p, p, C.c_int32, p, p, p]),
            "sclap_server_create": (C.c_int, [p, p, p]),
            "sclap_server_submit": (C.c_int, [p, i64, p, p, p, p, i32, dbl, u64, p]),
            "sclap_server_poll": (C.c_int, [p, i64, i32, p, p, p, p]),
            "sclap_server_destroy": (C.c_int, [p]),
            "sclap_debug_inject": (C.c_int, [i64, i64, i32]),
            "sclap_check_build": (C.c_int, []),
            "sclap_check_selftest": (C.c_int, [p]),
            "sclap_get_tuning": (None, [p]),
            "sclap_set_tuning": (C.c_int, [p]),
            "sclap_autotune": (C.c_int, [i32, p, p, i32, i32, p, p]),
            "sclap_profile_enable": (None, [C.c_int]),
            "sclap_profile_reset": (None, []),
            "sclap_profile_read": (None, [p]),
            "sclap_profile_timeline": (None, [C.c_int]),
            "sclap_profile_dump": (C.c_int64, [p, C.c_int64]),
            "sclap_profile_phases": (C.c_int64, [p, C.c_int64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _handle = h
    return _handle


def load():
    """Loads libsclap.so (raises if it is missing)."""
    return _lib()


def check_build() -> bool:
    """True when the loaded library is the bounds-check build."""
    return _lib().sclap_check_build() == 1


def check_selftest(stream=None) -> None:
    """Bounds-check build only: one checked index in range, one refused
    (sclap_check_selftest, on `stream` or the default stream); raises
    SclapError otherwise."""
    _check(_lib().sclap_check_selftest(None if stream is None else _stream(stream)),
           "sclap_check_selftest")


def sclap_profile_enable(on: bool = True) -> None:
    _lib().sclap_profile_enable(1 if on else 0)


def sclap_profile_reset() -> None:
    _lib().sclap_profile_reset()


def sclap_profile_read() -> dict:
    p = Profile()
    _lib().sclap_profile_read(C.byref(p))
    return p.to_dict()


def sclap_profile_timeline(on: bool = True) -> None:
    _lib().sclap_profile_timeline(1 if on else 0)


def sclap_profile_dump() -> dict:
    """{kernel name: (launches, total ms)} since the last dump."""
    buf = C.create_string_buffer(1 << 20)
    _lib().sclap_profile_dump(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.rsplit(" ", 2)
        out[name] = (int(cnt), float(ms))
    return out


def default_config(**overrides) -> Config:
    c = Config()
    _lib().sclap_default_config(C.byref(c))
    for k, v in overrides.items():
        setattr(c, k, int(v))
    return c


def _check(rc: int, where: str, allow=(OK,)):
    if rc not in allow:
        raise SclapError(rc, where)
    return rc


def _np(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dp(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class Result:
    block: object          # numpy array (host API) or torch tensor (device API)
    cut: int
    max_block_weight: int
    status: int
    stats: Optional[dict] = None


# --------------------------------------------------------------- whole partitioner
def sclap_partition(row_ptr, col, node_w=None, edge_w=None, k=2, eps=0.03, seed=0,
                    cfg: Optional[Config] = None) -> Result:
    """Host arrays in, host block ids out (sclap_partition)."""
    rp = _np(row_ptr, np.int64)
    cl = _np(col, np.int32)
    nw = _np(node_w, np.int32)
    ew = _np(edge_w, np.int32)
    n = rp.size - 1
    blk = np.empty(n, np.int32)
    cut, mb = C.c_int64(), C.c_int64()
    st = Stats()
    rc = _lib().sclap_partition(n, _hp(rp), _hp(cl), _hp(nw), _hp(ew), int(k), float(eps),
                                int(seed) & (2**64 - 1), C.byref(cfg) if cfg else None,
                                _hp(blk), C.byref(cut), C.byref(mb), C.byref(st))
    _check(rc, "sclap_partition", allow=(OK, EINFEASIBLE))
    return Result(blk, cut.value, mb.value, rc, st.to_dict())


def sclap_partition_device(row_ptr, col, node_w=None, edge_w=None, k=2, eps=0.03, seed=0,
                           cfg: Optional[Config] = None, block_out=None, stream=None) -> Result:
    """CUDA tensors in, CUDA tensor of block ids out (sclap_partition_device)."""
    import torch
    n = row_ptr.numel() - 1
    if block_out is None:
        block_out = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    cut, mb = C.c_int64(), C.c_int64()
    st = Stats()
    rc = _lib().sclap_partition_device(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w),
                                       int(k), float(eps), int(seed) & (2**64 - 1),
                                       C.byref(cfg) if cfg else None, _dp(block_out),
                                       C.byref(cut), C.byref(mb), C.byref(st), _stream(stream))
    _check(rc, "sclap_partition_device", allow=(OK, EINFEASIBLE))
    return Result(block_out, cut.value, mb.value, rc, st.to_dict())


def _batch_descs(graphs: Sequence[dict], device: bool):
    """sclap_graph descriptors for a batch, the output arrays, and the arrays
    the descriptors point into (kept alive by the caller)."""
    descs = (GraphDesc * len(graphs))()
    keep = []
    outs = []
    for i, g in enumerate(graphs):
        d = descs[i]
        if device:
            import torch
            rp, cl = g["row_ptr"], g["col"]
            out = torch.empty(rp.numel() - 1, dtype=torch.int32, device=rp.device)
            d.n = rp.numel() - 1
            d.row_ptr, d.col = _dp(rp).value, _dp(cl).value
            d.node_w = _dp(g.get("node_w")).value if g.get("node_w") is not None else None
            d.edge_w = _dp(g.get("edge_w")).value if g.get("edge_w") is not None else None
            d.block_out = _dp(out).value
            keep.append((rp, cl, g.get("node_w"), g.get("edge_w")))
        else:
            rp, cl = _np(g["row_ptr"], np.int64), _np(g["col"], np.int32)
            nw, ew = _np(g.get("node_w"), np.int32), _np(g.get("edge_w"), np.int32)
            out = np.empty(rp.size - 1, np.int32)
            d.n = rp.size - 1
            d.row_ptr, d.col = _hp(rp).value, _hp(cl).value
            d.node_w = _hp(nw).value if nw is not None else None
            d.edge_w = _hp(ew).value if ew is not None else None
            d.block_out = _hp(out).value
            keep.append((rp, cl, nw, ew))
        d.k = int(g.get("k", 2))
        d.eps = float(g.get("eps", 0.03))
        d.seed = int(g.get("seed", 0)) & (2**64 - 1)
        outs.append(out)
    return descs, outs, keep


def sclap_partition_batch(graphs: Sequence[dict], cfg: Optional[Config] = None,
                          device: bool = False, stream=None):
    """Partitions many graphs in one call (sclap_partition_batch).

    Each entry: dict(row_ptr, col, node_w=None, edge_w=None, k, eps, seed); numpy
    arrays when device=False, CUDA tensors when device=True.  Returns a list
    of Result (block ids as numpy arrays or CUDA tensors).
    """
    descs, outs, keep = _batch_descs(graphs, device)
    rc = _lib().sclap_partition_batch(len(graphs), C.cast(descs, C.c_void_p),
                                      C.byref(cfg) if cfg else None, 1 if device else 0,
                                      _stream(stream) if device else None)
    res = [Result(outs[i], descs[i].cut, descs[i].max_block_weight, descs[i].status)
           for i in range(len(graphs))]
    _check(rc, "sclap_partition_batch", allow=(OK, EINFEASIBLE))
    del keep
    return res


# --------------------------------------------------------------- step entry points
def sclap_lp_round(mode, row_ptr, col, node_w, edge_w, label, W, bound, rkey, sub_rounds,
                   active_cur=None, active_next=None, stream=None) -> int:
    moved = C.c_int64()
    n = row_ptr.numel() - 1
    rc = _lib().sclap_lp_round(int(mode), n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w),
                               _dp(label), _dp(W), W.numel(), int(bound),
                               int(rkey) & (2**64 - 1), int(sub_rounds), _dp(active_cur),
                               _dp(active_next), C.byref(moved), _stream(stream))
    _check(rc, "sclap_lp_round")
    return moved.value


def sclap_cluster(row_ptr, col, node_w, edge_w, U, seed, level=0, cfg=None, stream=None):
    import torch
    n = row_ptr.numel() - 1
    label = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    rounds = C.c_int32()
    rc = _lib().sclap_cluster(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w), int(U),
                              int(seed) & (2**64 - 1), int(level), C.byref(cfg) if cfg else None,
                              _dp(label), C.byref(rounds), _stream(stream))
    _check(rc, "sclap_cluster")
    return label, rounds.value


def sclap_cluster_hierarchy(row_ptr, col, node_w, edge_w, U, stop_nodes, seed, cfg=None,
                            stream=None):
    """Clustering hierarchy without k (device tensors in): returns (community
    of each input node as a CUDA tensor, contractions kept, node counts per
    level, input first)."""
    import torch
    n = row_ptr.numel() - 1
    comm = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    levels = C.c_int32()
    cap = 65
    level_n = np.zeros(cap, dtype=np.int64)
    rc = _lib().sclap_cluster_hierarchy(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w),
                                        int(U), int(stop_nodes), int(seed) & (2**64 - 1),
                                        C.byref(cfg) if cfg else None, _dp(comm),
                                        C.byref(levels), _hp(level_n), cap, _stream(stream))
    _check(rc, "sclap_cluster_hierarchy")
    return comm, levels.value, [int(x) for x in level_n[:levels.value + 1]]


def sclap_contract(row_ptr, col, node_w, edge_w, label, stream=None):
    """Returns (cmap, row_ptr, col, node_w, edge_w) of the coarse graph (CUDA)."""
    import torch
    n = row_ptr.numel() - 1
    m = col.numel()
    dev = row_ptr.device
    cmap = torch.empty(n, dtype=torch.int32, device=dev)
    cnw = torch.empty(n, dtype=torch.int32, device=dev)
    crp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ccol = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    cew = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    nc, mc = C.c_int64(), C.c_int64()
    rc = _lib().sclap_contract(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w), _dp(label),
                               _dp(cmap), C.byref(nc), _dp(cnw), _dp(crp), _dp(ccol), _dp(cew),
                               C.byref(mc), _stream(stream))
    _check(rc, "sclap_contract")
    a, b = nc.value, mc.value
    return cmap, crp[:a + 1], ccol[:b], cnw[:a], cew[:b]


def sclap_initial_partition(row_ptr, col, node_w, edge_w, k, Lmax, avg, seed, level=0,
                            cfg=None, stream=None):
    import torch
    n = row_ptr.numel() - 1
    blk = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    cut, best = C.c_int64(), C.c_int32()
    rc = _lib().sclap_initial_partition(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w),
                                        int(k), int(Lmax), int(avg), int(seed) & (2**64 - 1),
                                        int(level), C.byref(cfg) if cfg else None, _dp(blk),
                                        C.byref(cut), C.byref(best), _stream(stream))
    _check(rc, "sclap_initial_partition")
    return blk, cut.value, best.value


def sclap_refine(row_ptr, col, node_w, edge_w, k, Lmax, block, seed, phase=PH_REFINE, level=0,
                 cfg=None, stream=None) -> int:
    rounds = C.c_int32()
    n = row_ptr.numel() - 1
    rc = _lib().sclap_refine(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w), int(k),
                             int(Lmax), int(seed) & (2**64 - 1), int(phase), int(level),
                             C.byref(cfg) if cfg else None, _dp(block), C.byref(rounds),
                             _stream(stream))
    _check(rc, "sclap_refine")
    return rounds.value


def sclap_cut(row_ptr, col, edge_w, block, stream=None) -> int:
    cut = C.c_int64()
    n = row_ptr.numel() - 1
    rc = _lib().sclap_cut(n, _dp(row_ptr), _dp(col), _dp(edge_w), _dp(block), C.byref(cut),
                          _stream(stream))
    _check(rc, "sclap_cut")
    return cut.value


# Largest k sclap_cut_static accepts (SCLAP_CUT_STATIC_MAX_K in sclap.h).
CUT_STATIC_MAX_K = 4096


def sclap_cut_static(row_ptr, col, node_w, edge_w, block, k, stream=None):
    """Cut and block weights (c(V_i), i < k) of ``block`` without any device
    allocation: the library works in a fixed device array of its own, so
    k <= CUT_STATIC_MAX_K and calls must not overlap in time.  Device
    tensors in; returns (cut, numpy int64[k])."""
    cut = C.c_int64()
    n = row_ptr.numel() - 1
    bw = np.zeros(max(int(k), 1), dtype=np.int64)
    rc = _lib().sclap_cut_static(n, _dp(row_ptr), _dp(col), _dp(node_w), _dp(edge_w), _dp(block),
                                 int(k), C.byref(cut), _hp(bw), _stream(stream))
    _check(rc, "sclap_cut_static")
    return cut.value, bw[:int(k)]


@dataclass
class Served:
    """Result of one served request."""
    block: np.ndarray
    cut: int
    max_block_weight: int
    status: int
    latency_ms: float


class Server:
    """Continuous-batching partition server (sclap_server_*).  Requests are
    host arrays; results come back through poll()."""

    def __init__(self, cfg: Optional[Config] = None, device_budget_bytes: int = 0,
                 workers: int = 0, max_batch: int = 0, linger_us: int = 0):
        opts = ServerOptions(int(device_budget_bytes), int(workers), int(max_batch),
                             int(linger_us))
        h = C.c_void_p()
        rc = _lib().sclap_server_create(C.byref(cfg) if cfg else None, C.byref(opts),
                                        C.byref(h))
        _check(rc, "sclap_server_create")
        self._h = h
        self._n = {}

    def submit(self, row_ptr, col, node_w=None, edge_w=None, k=2, eps=0.03, seed=0) -> int:
        rp = _np(row_ptr, np.int64)
        cl = _np(col, np.int32)
        nw = _np(node_w, np.int32)
        ew = _np(edge_w, np.int32)
        rid = C.c_int64()
        rc = _lib().sclap_server_submit(self._h, rp.size - 1, _hp(rp), _hp(cl), _hp(nw), _hp(ew),
                                        int(k), float(eps), int(seed) & (2**64 - 1),
                                        C.byref(rid))
        _check(rc, "sclap_server_submit")
        self._n[rid.value] = rp.size - 1
        return rid.value

    def poll(self, request_id: int, timeout_ms: int = -1) -> Optional[Served]:
        """The request's result, or None while it is pending.  Raises
        SclapError for a failed request (and for an unknown id)."""
        n = self._n.get(request_id, 1)
        blk = np.empty(max(n, 1), np.int32)
        cut, mb, lat = C.c_int64(), C.c_int64(), C.c_double()
        rc = _lib().sclap_server_poll(self._h, int(request_id), int(timeout_ms), _hp(blk),
                                      C.byref(cut), C.byref(mb), C.byref(lat))
        if rc == PENDING:
            return None
        self._n.pop(request_id, None)
        _check(rc, "sclap_server_poll", allow=(OK, EINFEASIBLE))
        return Served(blk[:n], cut.value, mb.value, rc, lat.value)

    def close(self):
        if self._h:
            _lib().sclap_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass


def sclap_profile_phases() -> np.ndarray:
    """Per-sub-round records since the last reset, shape (count, 7): run kind,
    round, colour class, nodes, arcs, propose ms, admission ms."""
    n = _lib().sclap_profile_phases(None, 0)
    out = np.zeros((max(n, 1), 7), dtype=np.float64)
    m = _lib().sclap_profile_phases(out.ctypes.data_as(C.c_void_p), n)
    return out[:min(n, m)]


def debug_inject(wait_limit: int = 0, probe_limit: int = 0, fail_allocs: int = 0) -> None:
    """Host-side fault injection (sclap_debug_inject); all zeros restores
    the defaults."""
    _check(_lib().sclap_debug_inject(int(wait_limit), int(probe_limit), int(fail_allocs)),
           "sclap_debug_inject")


def get_tuning() -> Tuning:
    t = Tuning()
    _lib().sclap_get_tuning(C.byref(t))
    return t


def set_tuning(**kw) -> Tuning:
    """Changes some launch choices (sclap_set_tuning); returns the setting."""
    t = get_tuning()
    for k, v in kw.items():
        setattr(t, k, int(v))
    _check(_lib().sclap_set_tuning(C.byref(t)), "sclap_set_tuning")
    return get_tuning()


def autotune(graphs: Sequence[dict], cfg: Optional[Config] = None, device: bool = True,
             reps: int = 3, stream=None) -> Tuning:
    """Picks and installs the launch tuning for this batch (sclap_autotune)."""
    descs, outs, keep = _batch_descs(graphs, device)
    out = Tuning()
    rc = _lib().sclap_autotune(len(graphs), C.cast(descs, C.c_void_p),
                               C.byref(cfg) if cfg else None,
                               1 if device else 0, int(reps), C.byref(out),
                               _stream(stream) if device else None)
    _check(rc, "sclap_autotune")
    del keep, outs
    return out

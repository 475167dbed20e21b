#!/usr/bin/env python
"""Benchmark of the GB300 SCLaP partitioner on the batched workload.

Workload (default): 512 independent graphs of uneven size partitioned in one
batched call: half R-MAT (scale uniform in 10..16, edge factor 8,
a,b,c,d = 0.57,0.19,0.19,0.05), half 2D random geometric graphs (n
log-uniform in 1k..64k), k uniform in {2,4,8,16}, eps = 0.03, seed 0.  A
step = one full multilevel partition of every graph (coarsening, initial
partitioning, uncoarsening, repair, cut), inputs already resident in HBM
(~1 GB of CSR, larger than L2, so no flush is needed between steps).

Prints one JSON line.  value = partitions/s of the whole job (all ranks).
Extra keys: sclap_edges_per_s (arcs swept by LP / step time),
plain_partitions_per_s (the same graphs, one call each, equal cuts checked),
roofline (LP propose sweep vs the measured HBM copy peak), cpu_baseline (the
oracle's round-synchronous variant on the host), e2e (host buffers through
the C ABI, copies included), serving (p50/p99 latency of Poisson request
streams through the server), clocks, gpu_launches.

--impl reference times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): replicas only -- each rank partitions its own batch
(different graph seeds); no data-path collective.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

# Algorithmic bytes of the LP propose sweep.  Per arc: col (4) + edge weight
# (4) + label gather (4); on a level of unit edge weights no weight is read
# (8).  Per node: sub-round list entry (4), row_ptr pair (16), slot id (4),
# own label (4), node weight (4), proposal target (4) and admission key (8)
# written.
ARC_BYTES = 12
ARC_BYTES_UNIT = 8
SECTOR_BYTES = 32     # one DRAM sector: the cost of a label gather that misses L2
NODE_BYTES = 44
FAMILIES = ["thread_deg_le16", "warp_deg_le128_cta128", "cta256_512", "hub_global_table"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "large", "huge", "serve", "cpu"],
                    help="batched: the 512-graph batch (default); large: R-MAT scale 22 and "
                         "RGG 2^22, one graph per call, both round drivers; huge: one R-MAT "
                         "graph of --scale (default 27, edge factor 24) generated on the "
                         "device, k = 16; serve: Poisson request streams of mixed R-MAT and "
                         "RGG graphs through the server; cpu: the CPU oracles (sequential "
                         "and round-synchronous) on one host core")
    ap.add_argument("--scale", type=int, default=27, help="R-MAT scale of --workload huge")
    ap.add_argument("--graph-rounds", action="store_true",
                    help="run each level's LP rounds as one CUDA graph (device-side loop)")
    ap.add_argument("--autotune", action="store_true",
                    help="batched: before the warm-up, pick the launch tuning for this batch "
                         "with sclap_autotune (results unchanged; the choice goes into "
                         "config); large: pick it per graph at k = 8 and report its gain")
    ap.add_argument("--tuning", default="",
                    help="comma-separated field=value launch-tuning settings applied with "
                         "sclap_set_tuning before the run, e.g. contract_merge=0 (results "
                         "unchanged; the setting goes into config)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--phases", action="store_true",
                    help="print per-sub-round propose/admission times grouped by run kind "
                         "and round (stderr)")
    ap.add_argument("--timeline", action="store_true",
                    help="after the timed steps, run one step with per-kernel timeline "
                         "events and print the table to stderr")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(count, seed):
    procs = min(16, os.cpu_count() or 1)
    return gg.batch_workload(count, seed, processes=procs)


def rank_seed(rank):
    """Each rank partitions its own batch (replicas, weak scaling)."""
    return rank


def max_over_ranks(x, ws, device=None):
    """Largest value of x over all ranks (a plain float when ws == 1)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_dict(count, ws):
    return {
        "workload": f"batched-{count}: half R-MAT scale U[10,16] ef 8 (0.57,0.19,0.19,0.05), "
                    "half 2D RGG n logU[1k,64k] r=0.55*sqrt(ln n/n); k U{2,4,8,16}; eps 0.03; "
                    "unit int32 weights; seed 0",
        "graphs_per_rank": count,
        "ranks": ws,
        "l2": "inputs ~1 GB per batch, larger than L2 (no flush)",
        "params": "l=10 LP rounds coarse/refine, f=18, coarsen to max(1000,60k), 16 IP trials, "
                  "8 colour classes",
    }


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms.

    Started before the warm-up (so nvidia-smi's own start-up, which takes
    driver locks, falls outside the timed region); mark() and stop() bound the
    timed window, and only samples stamped inside it are summarised (all of
    them when fewer than two fall inside)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = None
        self.t1 = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def mark(self):
        self.t0 = datetime.datetime.now()

    def stop(self):
        self.t1 = datetime.datetime.now()
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.f.name)

        def stamp(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                return None
        inside = [r for r in rows if self.t0 and stamp(r) and self.t0 <= stamp(r) <= self.t1]
        window = "timed region" if len(inside) >= 2 else "warm-up and timed region"
        rows = [r[1:] for r in (inside if len(inside) >= 2 else rows)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "window": window}


def traffic_for(kernel_src):
    """dram bytes per propose launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if d.get("lp_cu_sha256_16") != h:
        return None
    return d.get("bytes_per_arc"), d.get("note")


def oracle_rate(graphs, seconds, steps=None):
    """Round-synchronous oracle on the host: partitions graphs in order until
    `seconds` of CPU work (at least one graph).  Returns (partitions/s, n)."""
    import oracle as O
    t0 = time.perf_counter()
    done = 0
    for g, k, eps in graphs:
        O.partition(g, k, eps, seed=0, variant=O.SYNC)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return done / (time.perf_counter() - t0), done


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    graphs = workload(args.count, 0)
    import oracle as O
    O.build()
    # one step = the first 16 graphs of the batch (a bounded sample)
    sample = graphs[:16]
    for _ in range(args.warmup):
        for g, k, eps in sample[:2]:
            O.partition(g, k, eps, seed=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for g, k, eps in sample:
            O.partition(g, k, eps, seed=0)
    dt = time.perf_counter() - t0
    value = args.steps * len(sample) / dt
    line = {
        "impl": "reference", "metric": "partitions/s", "value": value, "unit": "partitions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(config_dict(args.count, 1),
                       sample="each step partitions the first 16 graphs of the batch (a "
                              "bounded sample: the whole batch takes the oracle ~12 s); "
                              "value = partitions/s over the sample"),
        "cpu_baseline": {"value": value, "unit": "partitions/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {len(sample)} graphs of the batch per step, "
                                   "round-synchronous oracle, single thread"},
        "e2e": {"value": value, "unit": "partitions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host's CPU model and core count, as the OS reports them."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware") and not model:
                model = line.split(":", 1)[1].strip()
            if key == "cpu part" and not model:
                model = "ARM part " + line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return {"model": model or platform.processor() or platform.machine(),
            "machine": platform.machine(), "nproc": os.cpu_count()}


def cpu_workload(args):
    """CPU baseline of the plan: the paper's sequential SCLaP (increasing-
    degree order, immediate moves, FIFO active-node queues) and the
    round-synchronous variant the GPU follows, both single-threaded oracles,
    on the single-graph workload (R-MAT scale 16, edge factor 8, k = 2,
    eps = 0.03), seeds 0-4: wall time best and median, mean cut; and
    partitions/s of both over a bounded sample of the 512-graph batch."""
    import oracle as O
    O.build()
    g = gg.rmat(16, 8, 0)
    out = {}
    for name, var in (("sequential", O.SEQ), ("synchronous", O.SYNC)):
        ts, cuts = [], []
        for seed in range(5):
            t0 = time.perf_counter()
            r = O.partition(g, 2, 0.03, seed=seed, variant=var)
            ts.append(time.perf_counter() - t0)
            cuts.append(r.cut)
        ts.sort()
        out[name] = {"best_s": ts[0], "median_s": ts[2], "mean_cut": float(np.mean(cuts)),
                     "cuts": cuts}
    batch = workload(512, 0)
    sample = batch[::16][:32]            # 32 graphs spread over the batch
    rates = {}
    for name, var in (("sequential", O.SEQ), ("synchronous", O.SYNC)):
        t0 = time.perf_counter()
        for bg, k, eps in sample:
            O.partition(bg, k, eps, seed=0, variant=var)
        rates[name] = len(sample) / (time.perf_counter() - t0)
    line = {
        "metric": "seconds per partition (CPU oracle, 1 thread)", "unit": "s",
        "higher_is_better": False, "data": "synthetic",
        "config": {"workload": "R-MAT scale 16 ef 8 (65,536 nodes), k = 2, eps 0.03, seeds 0-4; "
                               "and every 16th graph of the 512-graph batch (32 graphs)",
                   "threads": 1},
        "host": cpu_model(),
        "single_graph": out,
        "batch_sample_partitions_per_s": rates,
        "sync_over_seq_mean_cut": out["synchronous"]["mean_cut"] / out["sequential"]["mean_cut"],
    }
    print(json.dumps(line), flush=True)


KINDS = {1: "cluster", 2: "refine", 3: "ip-trial", 5: "ip-refine", 6: "repair"}


def print_phases(ph, steps):
    """Per-step totals of the sub-round records, by run kind and round."""
    if ph.size == 0:
        return
    print(f"sub-rounds per step: {len(ph) / steps:.0f} (GB/s at 12 B per arc, an upper "
          "bound on levels of unit edge weights)", file=sys.stderr)
    print(f"{'kind':10s} {'round':>5s} {'subs':>5s} {'nodes':>11s} {'arcs':>12s} "
          f"{'sweep_ms':>9s} {'adm_ms':>8s} {'GB/s':>7s}", file=sys.stderr)
    keys = sorted({(int(r[0]), int(r[1])) for r in ph})
    for kind, rnd in keys + [(k, -1) for k in sorted({int(r[0]) for r in ph})]:
        m = (ph[:, 0] == kind) & ((ph[:, 1] == rnd) | (rnd < 0))
        q = ph[m]
        nodes, arcs = q[:, 3].sum() / steps, q[:, 4].sum() / steps
        sw, ad = q[:, 5].sum() / steps, q[:, 6].sum() / steps
        gbs = (ARC_BYTES * arcs + NODE_BYTES * nodes) / (sw / 1e3) / 1e9 if sw else 0.0
        print(f"{KINDS.get(kind, kind):10s} {'all' if rnd < 0 else rnd:>5} {len(q) / steps:5.0f} "
              f"{nodes:11.0f} {arcs:12.0f} {sw:9.3f} {ad:8.3f} {gbs:7.0f}", file=sys.stderr)


def sweep_by_kind(ph, steps=1):
    """Per run kind (clustering, local search, initial partitioning, ...)
    from the library's sub-round records: nodes and arcs swept, propose time,
    SCLaP edges/s (arcs / propose time) and algorithmic GB/s at 12 B per arc
    (an upper bound on levels of unit edge weights) + 44 B per node."""
    out = {}
    if ph.size == 0:
        return out
    for kind in sorted({int(r[0]) for r in ph}):
        q = ph[ph[:, 0] == kind]
        nodes, arcs = q[:, 3].sum() / steps, q[:, 4].sum() / steps
        sw = q[:, 5].sum() / steps
        out[KINDS.get(kind, str(kind))] = {
            "sub_rounds": len(q) / steps, "nodes": nodes, "arcs": arcs, "sweep_ms": sw,
            "edges_per_s": arcs / (sw / 1e3) if sw else None,
            "gbs": (ARC_BYTES * arcs + NODE_BYTES * nodes) / (sw / 1e3) / 1e9 if sw else None}
    return out


def serve_stream(P, graphs, lam, count, ref_cuts, seed=0):
    """Open-loop Poisson stream through the server: ``count`` requests (the
    batch's graphs in order, cycling) with exponential gaps of mean 1/lam s,
    submitted on time by one thread while the main thread collects results
    in order.  Latency = submit to completion, measured by the server."""
    import threading
    rng = np.random.default_rng(np.random.SeedSequence([0x53525645, seed, count]))
    gaps = rng.exponential(1.0 / lam, size=count)
    ids = [None] * count
    ready = [threading.Event() for _ in range(count)]
    with P.Server() as srv:
        def feeder():
            t_next = time.perf_counter()
            for i in range(count):
                t_next += gaps[i]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                g, k, eps = graphs[i % len(graphs)]
                ids[i] = srv.submit(g.row_ptr, g.col, None, None, k, eps, 0)
                ready[i].set()
        th = threading.Thread(target=feeder)
        t0 = time.perf_counter()
        th.start()
        lat, same = [], True
        for i in range(count):
            ready[i].wait()
            r = srv.poll(ids[i], -1)
            lat.append(r.latency_ms)
            same &= r.cut == ref_cuts[i % len(graphs)]
        t1 = time.perf_counter()
        th.join()
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    return {"lambda_per_s": lam, "requests": count, "p50_ms": q(0.50), "p99_ms": q(0.99),
            "partitions_per_s": count / (t1 - t0), "offered_per_s": count / float(gaps.sum()),
            "equal_cut": bool(same)}


def serve_request(i, seed=0):
    """Request i of the serving mix: even i an R-MAT graph with scale
    uniform in 12..20 (edge factor 8), odd i a 2D RGG with 2^u nodes, u
    uniform in [12, 20]; k uniform in {2, 4, 8, 16, 32, 64}; eps uniform in
    {0.01, 0.03, 0.05}; a partition seed of its own.  (Graph, k, eps, seed)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x53455256, seed, i]))
    k = int(rng.choice([2, 4, 8, 16, 32, 64]))
    eps = float(rng.choice([0.01, 0.03, 0.05]))
    pseed = int(rng.integers(0, 2**31))
    if i % 2 == 0:
        g = gg.rmat(int(rng.integers(12, 21)), 8, seed=7000 + i)
    else:
        g = gg.rgg2d(int(round(2.0 ** rng.uniform(12, 20))), seed=7000 + i)
    return g, k, eps, pseed


def serve_workload(args):
    """C5-style serving: a pool of 96 requests of the serving mix, submitted
    as open-loop Poisson streams at 50 to 2000 requests/s through the server
    (host arrays, default options: 2 workers, 120 GiB admission budget); each
    result must equal the same request partitioned alone.  Reported per
    rate: p50/p99 latency from submit to completion and completed
    partitions/s; and the one-at-a-time rate of the same requests."""
    import threading
    import multiprocessing as mp
    import torch
    import paper_1402_3281_gb300 as P
    P.load()
    torch.cuda.set_device(0)
    pool_n = 96
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        reqs = pool.starmap(serve_request, [(i, 0) for i in range(pool_n)])
    sampler = ClockSampler(0)
    sampler.start()
    for g, k, eps, sd in reqs[:8]:                       # warm-up
        P.sclap_partition(g.row_ptr, g.col, k=k, eps=eps, seed=sd)
    torch.cuda.synchronize()
    sampler.mark()
    t0 = time.perf_counter()
    alone = [P.sclap_partition(g.row_ptr, g.col, k=k, eps=eps, seed=sd) for g, k, eps, sd in reqs]
    plain_s = time.perf_counter() - t0
    ref = [(r.cut, r.block) for r in alone]
    runs = []
    for lam in (50, 200, 500, 1000, 2000):
        count = int(min(384, max(96, 2 * lam)))
        rng = np.random.default_rng(np.random.SeedSequence([0x50535452, lam, count]))
        gaps = rng.exponential(1.0 / lam, size=count)
        ids = [None] * count
        ready = [threading.Event() for _ in range(count)]
        with P.Server() as srv:
            def feeder():
                t_next = time.perf_counter()
                for i in range(count):
                    t_next += gaps[i]
                    d = t_next - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    g, k, eps, sd = reqs[i % pool_n]
                    ids[i] = srv.submit(g.row_ptr, g.col, None, None, k, eps, sd)
                    ready[i].set()
            th = threading.Thread(target=feeder)
            s0 = time.perf_counter()
            th.start()
            lat, same = [], True
            for i in range(count):
                ready[i].wait()
                r = srv.poll(ids[i], -1)
                lat.append(r.latency_ms)
                c, b = ref[i % pool_n]
                same &= r.cut == c and bool(np.array_equal(r.block, b))
            s1 = time.perf_counter()
            th.join()
        lat.sort()
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
        runs.append({"lambda_per_s": lam, "requests": count, "p50_ms": q(0.50),
                     "p99_ms": q(0.99), "partitions_per_s": count / (s1 - s0),
                     "offered_per_s": count / float(gaps.sum()), "equal_to_alone": bool(same)})
    clocks = sampler.stop()
    best = max(r["partitions_per_s"] for r in runs)
    h2d = sum(g.row_ptr.nbytes + g.col.nbytes for g, _, _, _ in reqs) / pool_n
    line = {
        "metric": "partitions/s", "value": best, "unit": "partitions/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic", "dtype": "int32",
        "config": {"workload": "serving: open-loop Poisson streams at 50/200/500/1000/2000 "
                               "req/s over a pool of 96 requests (even: R-MAT scale U[12,20] ef 8, "
                               "odd: 2D RGG 2^U[12,20] nodes; k U{2,4,8,16,32,64}; eps "
                               "U{0.01,0.03,0.05}); host arrays through sclap_server_* (2 workers, "
                               "120 GiB admission budget)",
                   "pool_nodes": int(sum(g.n for g, _, _, _ in reqs)),
                   "pool_arcs": int(sum(g.arcs for g, _, _, _ in reqs))},
        "plain_partitions_per_s": pool_n / plain_s,
        "served_vs_plain": best / (pool_n / plain_s),
        "runs": runs,
        "e2e": {"value": best, "unit": "partitions/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(sum(4 * g.n for g, _, _, _ in reqs) / pool_n)},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def large_graphs():
    """The large single graphs: R-MAT scale 22 (4,194,304 nodes, edge factor
    16) and a 2D random geometric graph with 2^22 nodes, both seed 0."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(2) as pool:
        a = pool.apply_async(gg.rmat, (22, 16, 0))
        b = pool.apply_async(gg.rgg2d, (1 << 22, 0))
        return [("rmat22-ef16", a.get()), ("rgg2d-2^22", b.get())]


def large_workload(args):
    """One big graph per call, k in {2, 8, 32, 64}, seeds 0..4, under the
    host-driven and the CUDA-graph round drivers.  Every result is checked:
    balance (every block <= Lmax), the cut recounted independently on the
    device (sclap_cut), and equality between the two drivers."""
    import torch
    import paper_1402_3281_gb300 as P
    P.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sampler = ClockSampler(0)
    sampler.start()
    runs = []
    edges_total, ms_total = 0, {"host": 0.0, "graph": 0.0}
    all_ok = True
    rooflines, tuned = {}, {}
    default_tuning = P.get_tuning().to_dict()

    def median_ms(rp, col, k, reps=3):
        ms = []
        for _ in range(reps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            P.sclap_partition_device(rp, col, k=k, eps=0.03, seed=0)
            a1.record(stream)
            torch.cuda.synchronize()
            ms.append(a0.elapsed_time(a1))
        return sorted(ms)[len(ms) // 2]

    for name, g in large_graphs():
        rp, col = t(g.row_ptr), t(g.col)
        if args.autotune:
            # sclap_autotune on this graph at k = 8; its choice is used for
            # every run of the graph, and its gain reported
            P.set_tuning(**default_tuning)
            P.sclap_partition_device(rp, col, k=8, eps=0.03, seed=0)
            before = median_ms(rp, col, 8)
            tu = P.autotune([dict(row_ptr=rp, col=col, k=8, eps=0.03, seed=0)], reps=3)
            after = median_ms(rp, col, 8)
            tuned[name] = {"tuning": tu.to_dict(), "ms_default": before, "ms_tuned": after,
                           "gain": before / after if after > 0 else None}
        for k in (2, 8, 32, 64):
            for seed in range(5):
                res = {}
                for drv, gr in (("host", 0), ("graph", 1)):
                    cfg = P.default_config(graph_rounds=gr)
                    if seed == 0:      # warm-up for this shape
                        P.sclap_partition_device(rp, col, k=k, eps=0.03, seed=seed, cfg=cfg)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    if drv == "host" and not runs:
                        sampler.mark()
                    e0.record(stream)
                    r = P.sclap_partition_device(rp, col, k=k, eps=0.03, seed=seed, cfg=cfg)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    res[drv] = (r, e0.elapsed_time(e1))
                rh, mh = res["host"]
                rg, mg = res["graph"]
                Lmax = int(rh.stats["Lmax"])
                bw = torch.bincount(rh.block.long(), minlength=k)
                ok = (rh.status == 0 and int(bw.max()) <= Lmax
                      and P.sclap_cut(rp, col, None, rh.block) == rh.cut
                      and rg.cut == rh.cut and bool(torch.equal(rg.block, rh.block)))
                all_ok &= ok
                edges_total += g.edges
                ms_total["host"] += mh
                ms_total["graph"] += mg
                runs.append({"graph": name, "k": k, "seed": seed, "cut": rh.cut,
                             "ms_host": mh, "ms_graph": mg, "levels": rh.stats["levels"],
                             "checked": ok})
        # the propose sweep's roofline on this graph: one more call (k = 8,
        # seed 0, host driver) with CUDA events around every propose phase
        P.sclap_profile_reset()
        P.sclap_profile_enable(True)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        P.sclap_partition_device(rp, col, k=8, eps=0.03, seed=0)
        p1.record(stream)
        torch.cuda.synchronize()
        P.sclap_profile_enable(False)
        rf = propose_roofline(P.sclap_profile_read(), p0.elapsed_time(p1), 1)
        rooflines[name] = {x: rf[x] for x in ("achieved", "peak", "unit", "frac",
                                              "avg_launch_ms", "launches", "share_of_step")}
    P.set_tuning(**default_tuning)
    clocks = sampler.stop()
    line = {
        "metric": "input edges/s", "value": edges_total / (ms_total["host"] / 1000.0),
        "unit": "edges/s", "n_gpus": 1, "higher_is_better": True,
        "data": "synthetic",
        "config": {"workload": "large single graphs: R-MAT scale 22 ef 16 (a,b,c,d = "
                               "0.57,0.19,0.19,0.05) and 2D RGG 2^22 nodes r=0.55*sqrt(ln n/n); "
                               "k in {2,8,32,64}, eps 0.03, seeds 0-4, one graph per call"},
        "graph_driver_value": edges_total / (ms_total["graph"] / 1000.0),
        "all_checked": bool(all_ok), "runs": runs, "clocks": clocks,
        "propose_roofline_k8": rooflines,
    }
    if args.autotune:
        line["autotuned"] = tuned
    print(json.dumps(line), flush=True)


def propose_roofline(prof, prof_ms, steps):
    """Roofline of the LP propose sweep from the library's profile of `steps`
    profiled calls taking prof_ms in all: algorithmic bytes of every propose
    phase over their fork-to-join time, against the measured HBM peak."""
    swept = sum(prof["propose_arcs"])
    unit_arcs = prof["propose_arcs_unit"]
    prop_ms = prof["sweep_ms"]
    prop_bytes = (ARC_BYTES * (swept - unit_arcs) + ARC_BYTES_UNIT * unit_arcs
                  + NODE_BYTES * sum(prof["propose_nodes"]))
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = prop_bytes / (prop_ms / 1000.0) / 1e9 if prop_ms > 0 else 0.0
    # the same phases with every label gather counted as the 32-byte sector
    # it touches (what it costs once the label array no longer fits in L2)
    sec_bytes = prop_bytes + (SECTOR_BYTES - 4) * swept
    achieved_sec = sec_bytes / (prop_ms / 1000.0) / 1e9 if prop_ms > 0 else 0.0
    tr = traffic_for(os.path.join(ROOT, "paper_1402_3281_gb300", "csrc", "lp.cu"))
    nl = prof["sweeps"]
    return {
        "kernel": "LP propose sweep of a sub-round (k_propose_small, k_propose_warp, "
                  "k_propose_blk*: the degree-bucket launches of one colour class, run "
                  "concurrently); one 'launch' = one such phase, timed fork to join with "
                  "CUDA events",
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "bytes_model": "12 B per scanned arc (8 on levels of unit edge weights) + 44 B per "
                       "listed node",
        "arcs_unit_weight": unit_arcs,
        "frac": achieved / peak, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
        "sector_model": {"achieved": achieved_sec, "frac": achieved_sec / peak,
                         "bytes": "as above with each label gather at 32 B (one sector)"},
        "traffic": (tr[0] * swept / nl if tr and tr[0] else None) if nl else None,
        "bytes_per_launch": prop_bytes / nl if nl else None,
        "avg_launch_ms": prop_ms / nl if nl else None,
        "launches": nl,
        "share_of_step": prop_ms / prof_ms if prof_ms else None,
        "profiled_ms_per_step": prof_ms / steps,
        "per_family": {FAMILIES[b]: {"ms": prof["propose_ms"][b], "launches": prof["propose_launches"][b],
                                     "nodes": prof["propose_nodes"][b], "arcs": prof["propose_arcs"][b]}
                       for b in range(4)},
    }


def huge_workload(args):
    """One R-MAT graph of 2^scale nodes and edge factor 24, generated on the
    device (graphgen.device: same model as the host generator, counter-based
    draws), partitioned with k = 16 after a warm-up on a scale-16 graph.  The
    result is checked (balance, a device recount of the cut); a run that does
    not fit in device memory reports the library's out-of-memory error."""
    import torch
    import paper_1402_3281_gb300 as P
    from graphgen.device import rmat_torch
    P.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rp_w, col_w = rmat_torch(16, 24, 1, device=dev)
    P.sclap_partition_device(rp_w, col_w, k=16, eps=0.03, seed=0)
    t0 = time.perf_counter()
    try:
        rp, col = rmat_torch(args.scale, 24, 0, device=dev)
    except torch.cuda.OutOfMemoryError as e:
        print(json.dumps({"metric": "input edges/s", "unit": "edges/s", "n_gpus": 1,
                          "higher_is_better": True, "data": "synthetic", "value": None,
                          "config": {"workload": f"R-MAT scale {args.scale} ef 24, generated on "
                                                 "the device, k = 16"},
                          "error": "generation: " + str(e).splitlines()[0]}), flush=True)
        return
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n, arcs = rp.numel() - 1, col.numel()
    del rp_w, col_w
    torch.cuda.empty_cache()
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    line = {"metric": "input edges/s", "unit": "edges/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": f"R-MAT scale {args.scale} ef 24 (a,b,c,d = 0.57,0.19,0.19,0.05), "
                                   "generated on the device, k = 16, eps 0.03, seed 0, one call",
                       "n": n, "arcs": arcs, "generation_s": gen_s}}
    try:
        e0.record(stream)
        res = P.sclap_partition_device(rp, col, k=16, eps=0.03, seed=0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bw = torch.bincount(res.block.long(), minlength=16)
        ok = (res.status == 0 and int(bw.max()) <= int(res.stats["Lmax"])
              and P.sclap_cut(rp, col, None, res.block) == res.cut)
        st = res.stats
        line.update(value=(arcs // 2) / (ms / 1000.0), ms=ms, cut=res.cut,
                    levels=st["levels"], level_n=st["level_n"], level_m=st["level_m"],
                    cluster_rounds=st.get("cluster_rounds"), ip_cut=st.get("ip_cut"),
                    checked=bool(ok))
    except P.SclapError as e:
        line.update(value=None, error=str(e),
                    torch_reserved_gb=torch.cuda.memory_reserved() / 1e9)
    line["clocks"] = sampler.stop()
    if line.get("value"):
        # one more call with CUDA events around every propose phase: the
        # sweep's roofline at this size
        P.sclap_profile_reset()
        P.sclap_profile_enable(True)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        P.sclap_partition_device(rp, col, k=16, eps=0.03, seed=0)
        p1.record(stream)
        torch.cuda.synchronize()
        P.sclap_profile_enable(False)
        line["roofline"] = propose_roofline(P.sclap_profile_read(), p0.elapsed_time(p1), 1)
        line["sweep_by_kind"] = sweep_by_kind(P.sclap_profile_phases())
    if args.timeline and line.get("value"):
        # one more call with an event after every launch: time per kernel
        P.sclap_profile_dump()
        P.sclap_profile_timeline(True)
        P.sclap_partition_device(rp, col, k=16, eps=0.03, seed=0)
        torch.cuda.synchronize()
        P.sclap_profile_timeline(False)
        tl = P.sclap_profile_dump()
        tot = sum(v[1] for v in tl.values())
        print(f"timeline of one call: {tot:.2f} ms", file=sys.stderr)
        for name, (cnt, ms) in sorted(tl.items(), key=lambda x: -x[1][1]):
            print(f"  {name:28s} {cnt:7d} {ms:10.3f} ms {100 * ms / tot:6.1f}%", file=sys.stderr)
    print(json.dumps(line), flush=True)


def apply_tuning(args):
    if not args.tuning or args.impl == "reference" or args.workload == "cpu":
        return
    import paper_1402_3281_gb300 as P
    P.load()
    kv = dict(item.split("=", 1) for item in args.tuning.split(",") if item)
    P.set_tuning(**{k.strip(): int(v) for k, v in kv.items()})


def main():
    args = parse()
    apply_tuning(args)
    if args.workload == "large":
        large_workload(args)
        return
    if args.workload == "huge":
        huge_workload(args)
        return
    if args.workload == "serve":
        serve_workload(args)
        return
    if args.workload == "cpu":
        cpu_workload(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    ws, rank, local = dist_env()
    graphs = workload(args.count, rank_seed(rank))

    import torch
    import paper_1402_3281_gb300 as P
    P.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    items = [dict(row_ptr=t(g.row_ptr), col=t(g.col), k=k, eps=eps, seed=0)
             for g, k, eps in graphs]
    arcs_in = sum(g.arcs for g, _, _ in graphs)
    torch.cuda.synchronize()

    cfg = P.default_config(graph_rounds=1 if args.graph_rounds else 0)
    tuning = P.autotune(items, cfg=cfg, reps=3) if args.autotune else P.get_tuning()
    sampler = ClockSampler(local)
    sampler.start()
    ref = None
    for _ in range(args.warmup):
        ref = P.sclap_partition_batch(items, cfg=cfg, device=True)
    torch.cuda.synchronize()
    ref_cuts = [r.cut for r in ref]

    # timed steps: no event instrumentation inside (only the launch counter)
    P.sclap_profile_enable(False)
    P.sclap_profile_reset()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler.mark()
    e0.record(stream)
    last = None
    for _ in range(args.steps):
        last = P.sclap_partition_batch(items, cfg=cfg, device=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = P.sclap_profile_read()["kernel_launches"]
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    # the same steps again with CUDA events around every propose phase (the
    # roofline's time base) and launch
    P.sclap_profile_reset()
    P.sclap_profile_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(args.steps):
        P.sclap_partition_batch(items, cfg=cfg, device=True)
    p1.record(stream)
    torch.cuda.synchronize()
    P.sclap_profile_enable(False)
    prof = P.sclap_profile_read()
    prof_ms = p0.elapsed_time(p1)
    if args.phases:
        print_phases(P.sclap_profile_phases(), args.steps)
    if args.timeline:
        P.sclap_profile_dump()
        P.sclap_profile_timeline(True)
        P.sclap_partition_batch(items, device=True)
        torch.cuda.synchronize()
        P.sclap_profile_timeline(False)
        tl = P.sclap_profile_dump()
        tot = sum(v[1] for v in tl.values())
        print(f"timeline of one step: {tot:.2f} ms", file=sys.stderr)
        for name, (cnt, ms) in sorted(tl.items(), key=lambda x: -x[1][1]):
            print(f"  {name:28s} {cnt:7d} {ms:10.3f} ms {100 * ms / tot:6.1f}%", file=sys.stderr)
    deterministic = [r.cut for r in last] == ref_cuts
    balanced = all(r.status == 0 for r in last)

    parts = args.steps * len(graphs) * ws
    value = parts / (elapsed_ms / 1000.0)
    swept = sum(prof["propose_arcs"])
    roofline = propose_roofline(prof, prof_ms, args.steps)

    conf = config_dict(len(graphs), ws)
    conf["lp_rounds_driver"] = "cuda-graph (WHILE node per level)" if args.graph_rounds else "host"
    conf["launch_tuning"] = dict(tuning.to_dict(), autotuned=bool(args.autotune))
    line = {
        "metric": "partitions/s", "value": value, "unit": "partitions/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": conf,
        "sclap_edges_per_s": swept / (elapsed_ms / 1000.0) * (ws if ws > 1 else 1),
        "input_edges_per_s": arcs_in / 2 * args.steps * ws / (elapsed_ms / 1000.0),
        "deterministic": deterministic, "balanced": balanced,
        "roofline": roofline, "clocks": clocks,
        "gpu_launches": launches,
    }

    if rank == 0 and not args.no_plain:
        # the same graphs, one call each (the plain form), and equal cuts
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = [P.sclap_partition_device(it["row_ptr"], it["col"], k=it["k"], eps=it["eps"],
                                          seed=0) for it in items]
        torch.cuda.synchronize()
        pt = time.perf_counter() - t0
        line["plain_partitions_per_s"] = len(items) / pt
        line["batched_vs_plain"] = value / ws / (len(items) / pt)
        line["equal_cut"] = [p.cut for p in plain] == ref_cuts

    if not args.no_e2e:
        host_items = [dict(row_ptr=g.row_ptr, col=g.col, k=k, eps=eps, seed=0)
                      for g, k, eps in graphs]
        h2d = sum(g.row_ptr.nbytes + g.col.nbytes for g, _, _ in graphs)
        d2h = sum(4 * g.n for g, _, _ in graphs)
        # one untimed call first, as for the device-resident steps (the
        # library's host staging buffer is allocated on first use)
        P.sclap_partition_batch(host_items, device=False)
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(2, args.steps))
        for _ in range(e2e_steps):
            hres = P.sclap_partition_batch(host_items, device=False)
        torch.cuda.synchronize()
        et = max_over_ranks(time.perf_counter() - t0, ws, dev)
        line["e2e"] = {"value": e2e_steps * len(graphs) * ws / et, "unit": "partitions/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "equal_cut": [r.cut for r in hres] == ref_cuts}

    if rank == 0 and not args.no_single:
        # one graph, one call: R-MAT scale 16 (65,536 nodes), edge factor 8,
        # k = 2, eps = 0.03, seed 0 -- device-resident, latency per call
        g1 = gg.rmat(16, 8, 0)
        rp1, col1 = t(g1.row_ptr), t(g1.col)
        for _ in range(3):
            P.sclap_partition_device(rp1, col1, k=2, eps=0.03, seed=0)
        torch.cuda.synchronize()
        lat = []
        for _ in range(10):
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            r1 = P.sclap_partition_device(rp1, col1, k=2, eps=0.03, seed=0)
            q1.record(stream)
            torch.cuda.synchronize()
            lat.append(q0.elapsed_time(q1))
        lat.sort()
        line["single_graph"] = {
            "workload": "R-MAT scale 16 ef 8 (65,536 nodes, %d undirected edges), k=2, eps=0.03, "
                        "seed 0, device arrays, one call" % g1.edges,
            "ms_median": lat[len(lat) // 2], "ms_min": lat[0],
            "input_edges_per_s": g1.edges / (lat[len(lat) // 2] / 1000.0),
            "cut": r1.cut, "levels": r1.stats["levels"]}

    if rank == 0 and not args.no_serve:
        runs = [serve_stream(P, graphs, lam, cnt, ref_cuts)
                for lam, cnt in ((50, 100), (500, len(graphs)), (2000, len(graphs)))]
        line["serving"] = {
            "workload": "open-loop Poisson stream of this batch's graphs (in order), "
                        "host arrays, sclap_server_* with default options (2 workers, "
                        "120 GiB admission budget, batches up to 512)",
            "runs": runs}

    if rank == 0 and ws == 1:
        rate, done = oracle_rate(graphs, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "partitions/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {done} graphs of the batch in order "
                                          f"(~{args.cpu_seconds:.0f} s), round-synchronous "
                                          "oracle, single thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

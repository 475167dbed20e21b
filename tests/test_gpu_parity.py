"""GPU parity: every step of the CUDA path, called through the C ABI, equals the
CPU oracle's round-synchronous variant bit for bit (labels, weights, coarse
graphs, blocks, cuts).  Inputs are seeded synthetic graphs spanning every
degree bucket of the LP sweep (lane groups, warp / CTA shared-memory tables,
global-memory tables for hubs) and both admission paths (all-pairs and radix
select).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1402_3281_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


def dt(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).to(DEV)


def dg(g):
    return dt(g.row_ptr), dt(g.col), dt(g.node_w), dt(g.edge_w)


def hub_graph(seed=0):
    """R-MAT plus a star whose centre has degree 9000 (global-table bucket)."""
    base = gg.rmat(12, 8, seed)
    n = base.n
    src = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = src < base.col
    s = np.concatenate([src[keep], np.zeros(9000, np.int64)])
    d = np.concatenate([base.col[keep], np.arange(n, n + 9000)])
    s = np.concatenate([s, np.arange(n, n + 9000)])
    d = np.concatenate([d, np.repeat(np.arange(1, 100), 91)[:9000]])
    return gg.from_edges(n + 9000, s, d, name="hub")


def split_hub_graph(seed=0):
    """R-MAT with two hubs whose rows span several accumulation parts
    (16,384 arcs each): node 0 joined to 40,000 new leaves, node 1 to the
    last 20,000 of them; every leaf also meets one of nodes 2..200.  Random
    node and edge weights."""
    base = gg.rmat(12, 8, seed)
    n, L = base.n, 40000
    src = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = src < base.col
    leaves = np.arange(n, n + L)
    s = np.concatenate([src[keep], np.zeros(L, np.int64), np.ones(L // 2, np.int64), leaves])
    d = np.concatenate([base.col[keep], leaves, leaves[L // 2:], 2 + np.arange(L) % 199])
    g = gg.from_edges(n + L, s, d, name="split-hub")
    return gg.random_weights(g, seed + 5, max_node_w=3, max_edge_w=5)


GRAPHS = {
    "rmat12": lambda: gg.rmat(12, 8, 1),
    "rmat16": lambda: gg.rmat(16, 8, 0),
    "rgg": lambda: gg.rgg2d(5000, 2),
    "weighted": lambda: gg.random_weights(gg.rmat(11, 8, 4), 7, max_node_w=5, max_edge_w=9),
    "star": lambda: gg.star(3000),
    "hub": lambda: hub_graph(2),
    "split_hub": lambda: split_hub_graph(3),
}


@pytest.fixture(scope="module", params=sorted(GRAPHS))
def graph(request):
    return GRAPHS[request.param]()


# ------------------------------------------------------------------ one round
@pytest.mark.parametrize("S", [1, 3, 8])
def test_cluster_round_bit_exact(graph, S):
    rng = np.random.default_rng(S)
    g = graph
    label = np.arange(g.n, dtype=np.int32)
    if S == 3:  # start from a partial clustering so some clusters are near the bound
        label = (np.arange(g.n) // 3).astype(np.int32)
    W = np.bincount(label, weights=g.node_w, minlength=g.n).astype(np.int64)
    U = int(W.max()) + int(rng.integers(2, 40))
    rkey = int(rng.integers(1, 2**62))
    ol, oW, om, on = O.lp_round(g, O.MODE_CLUSTER, label, W, U, rkey, S, want_next=True)
    rp, col, nw, ew = dg(g)
    tl, tW = dt(label), dt(W)
    an = torch.zeros(g.n, dtype=torch.uint8, device=DEV)
    moved = P.sclap_lp_round(0, rp, col, nw, ew, tl, tW, U, rkey, S, active_next=an)
    assert moved == om
    assert np.array_equal(tl.cpu().numpy(), ol)
    assert np.array_equal(tW.cpu().numpy(), oW)
    assert np.array_equal(an.cpu().numpy(), on)


@pytest.mark.parametrize("k", [2, 7, 64])
def test_refine_round_bit_exact(graph, k):
    rng = np.random.default_rng(k)
    g = graph
    label = rng.integers(0, k, g.n).astype(np.int32)
    if k == 7:  # overload block 0 so forced moves and the source cap run
        label[rng.random(g.n) < 0.3] = 0
    W = np.bincount(label, weights=g.node_w, minlength=k).astype(np.int64)
    Lmax = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), k, 0.03)[0]
    active = (rng.random(g.n) < 0.7).astype(np.uint8)
    rkey = int(rng.integers(1, 2**62))
    ol, oW, om, on = O.lp_round(g, O.MODE_REFINE, label, W, Lmax, rkey, 8, active_cur=active,
                                want_next=True)
    rp, col, nw, ew = dg(g)
    tl, tW = dt(label), dt(W)
    an = torch.zeros(g.n, dtype=torch.uint8, device=DEV)
    moved = P.sclap_lp_round(1, rp, col, nw, ew, tl, tW, Lmax, rkey, 8, active_cur=dt(active),
                             active_next=an)
    assert moved == om
    assert np.array_equal(tl.cpu().numpy(), ol)
    assert np.array_equal(tW.cpu().numpy(), oW)
    assert np.array_equal(an.cpu().numpy(), on)


def test_large_overflow_segment_uses_radix_select():
    # Every leaf of a 5000-leaf star proposes the centre's cluster: one
    # segment far above the all-pairs limit.
    g = gg.star(5000)
    label = np.arange(g.n, dtype=np.int32)
    W = np.ones(g.n, np.int64)
    for U, S in [(17, 1), (1500, 1), (2600, 2)]:
        ol, oW, om, _ = O.lp_round(g, O.MODE_CLUSTER, label, W, U, 77, S)
        rp, col, nw, ew = dg(g)
        tl, tW = dt(label), dt(W)
        moved = P.sclap_lp_round(0, rp, col, nw, ew, tl, tW, U, 77, S)
        assert moved == om
        assert np.array_equal(tl.cpu().numpy(), ol)
        assert np.array_equal(tW.cpu().numpy(), oW)


# ------------------------------------------------------------------ level steps
def test_cluster_level_bit_exact(graph):
    g = graph
    Lmax, U = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), 2, 0.03)
    ol, orounds = O.cluster(g, U, seed=11, level=2)
    tl, rounds = P.sclap_cluster(*dg(g), U, 11, 2)
    assert rounds == orounds
    assert np.array_equal(tl.cpu().numpy(), ol)


def test_cluster_level_active_nodes_bit_exact(graph):
    """Active nodes during coarsening (configuration A)."""
    g = graph
    Lmax, U = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), 2, 0.03)
    ol, orounds = O.cluster(g, U, seed=5, level=1, cfg=O.config(cluster_active=1))
    tl, rounds = P.sclap_cluster(*dg(g), U, 5, 1, cfg=P.default_config(cluster_active=1))
    assert rounds == orounds
    assert np.array_equal(tl.cpu().numpy(), ol)


@pytest.mark.parametrize("U,stop,active", [(30, 100, 0), (400, 1, 0), (60, 1, 1)])
def test_cluster_hierarchy_bit_exact(graph, U, stop, active):
    """Clustering-only hierarchy (no k): communities and level sizes."""
    g = graph
    oc, olev, osz = O.cluster_hierarchy(g, U, stop, 13, cfg=O.config(cluster_active=active))
    tc, tlev, tsz = P.sclap_cluster_hierarchy(*dg(g), U, stop, 13,
                                              cfg=P.default_config(cluster_active=active))
    assert (tlev, tsz) == (olev, osz)
    assert np.array_equal(tc.cpu().numpy(), oc)


def test_cluster_hierarchy_edge_cases():
    g = gg.clique_ring(20, 8)
    tc, tlev, tsz = P.sclap_cluster_hierarchy(*dg(g), 8, 1, 2)
    oc, olev, osz = O.cluster_hierarchy(g, 8, 1, 2)
    assert (tlev, tsz) == (olev, osz) == (1, [160, 20])
    assert np.array_equal(tc.cpu().numpy(), oc)
    g = gg.from_edges(500, [], [])                   # no edges: nothing to merge
    tc, tlev, _ = P.sclap_cluster_hierarchy(*dg(g), 10, 1, 0)
    assert tlev == 0 and np.array_equal(tc.cpu().numpy(), np.arange(500))
    with pytest.raises(P.SclapError):                # U must be >= 1
        P.sclap_cluster_hierarchy(*dg(g), 0, 1, 0)


def _canon(rp, col, w):
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    o = np.lexsort((col, src))
    return src[o], col[o], w[o]


def test_contract_bit_exact(graph):
    g = graph
    U = 25
    lab, _ = O.cluster(g, U, seed=3)
    for label in (lab, np.arange(g.n, dtype=np.int32),
                  np.random.default_rng(1).integers(0, max(1, g.n // 50), g.n).astype(np.int32)):
        c = O.contract(g, label)
        cmap, crp, ccol, cnw, cew = P.sclap_contract(*dg(g), dt(label))
        assert np.array_equal(cmap.cpu().numpy(), c.cmap)
        assert np.array_equal(cnw.cpu().numpy(), c.node_w)
        assert np.array_equal(crp.cpu().numpy(), c.row_ptr)
        a = _canon(crp.cpu().numpy(), ccol.cpu().numpy(), cew.cpu().numpy())
        b = _canon(c.row_ptr, c.col, c.edge_w)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("k", [2, 5, 16])
def test_initial_partition_bit_exact(k):
    for g in (gg.rgg2d(1500, 3), gg.random_weights(gg.rmat(10, 8, 2), 3), gg.path(300)):
        cV = int(g.node_w.sum())
        Lmax, _ = O.bounds(cV, int(g.node_w.max()), k, 0.03)
        avg = -(-cV // k)
        cfg_o = O.config(ip_trials=6)
        ob, ocut, obest = O.initial_partition(g, k, Lmax, avg, seed=9, level=3, cfg=cfg_o)
        cfg = P.default_config(ip_trials=6)
        tb, cut, best = P.sclap_initial_partition(*dg(g), k, Lmax, avg, 9, 3, cfg=cfg)
        assert (cut, best) == (ocut, obest)
        assert np.array_equal(tb.cpu().numpy(), ob)


def test_ggg_single_trial_bit_exact():
    # one trial with no LP afterwards: the growing + water-filling step alone
    g = gg.random_weights(gg.rgg2d(2000, 5), 2)
    g = gg.Graph(g.row_ptr, g.col, g.node_w, g.edge_w)
    k = 6
    cV = int(g.node_w.sum())
    avg = -(-cV // k)
    Lmax = 10**9   # no local search moves can happen... (bound irrelevant, rounds = 0)
    cfg_o = O.config(ip_trials=1, lp_rounds_refine=0)
    ob, ocut, _ = O.initial_partition(g, k, Lmax, avg, seed=5, level=0, cfg=cfg_o)
    tb, cut, _ = P.sclap_initial_partition(*dg(g), k, Lmax, avg, 5, 0,
                                           cfg=P.default_config(ip_trials=1, lp_rounds_refine=0))
    assert cut == ocut
    assert np.array_equal(tb.cpu().numpy(), ob)


def test_refine_level_bit_exact(graph):
    g = graph
    k = 4
    rng = np.random.default_rng(5)
    blk = rng.integers(0, k, g.n).astype(np.int32)
    Lmax = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), k, 0.03)[0]
    ob, orounds = O.refine(g, k, Lmax, blk, seed=21, phase=O.PH_REFINE, level=1)
    tb = dt(blk)
    rounds = P.sclap_refine(*dg(g), k, Lmax, tb, 21, O.PH_REFINE, 1)
    assert rounds == orounds
    assert np.array_equal(tb.cpu().numpy(), ob)


def test_cut_matches_oracle(graph):
    g = graph
    rng = np.random.default_rng(0)
    for k in (2, 9):
        b = rng.integers(0, k, g.n).astype(np.int32)
        rp, col, nw, ew = dg(g)
        assert P.sclap_cut(rp, col, ew, dt(b)) == O.cut(g, b)


# ------------------------------------------------------------------ end to end
E2E = [
    ("rmat16", 2), ("rmat16", 8), ("rmat12", 4), ("rgg", 2), ("rgg", 16), ("weighted", 3),
    ("star", 2), ("hub", 4), ("split_hub", 8), ("split_hub", 64),
]


@pytest.mark.parametrize("name,k", E2E)
def test_partition_bit_exact(name, k):
    g = GRAPHS[name]()
    ref = O.partition(g, k, 0.03, seed=0)
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=0)
    assert res.status == ref.status
    assert res.cut == ref.cut
    assert np.array_equal(res.block.cpu().numpy(), ref.block)
    assert res.max_block_weight == ref.max_block_weight
    st = res.stats
    assert st["levels"] == ref.stats.levels
    assert st["level_n"] == list(ref.stats.level_n[:ref.stats.levels])


@pytest.mark.parametrize("name", ["rmat16", "rgg", "weighted"])
def test_partition_active_coarsening_bit_exact(name):
    g = GRAPHS[name]()
    ref = O.partition(g, 8, 0.03, seed=2, cfg=O.config(cluster_active=1))
    res = P.sclap_partition_device(*dg(g), k=8, eps=0.03, seed=2,
                                   cfg=P.default_config(cluster_active=1))
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)
    assert res.stats["level_n"] == list(ref.stats.level_n[:ref.stats.levels])


@pytest.mark.parametrize("gname,k", [("split_hub", 1500), ("rmat14", 1100)])
def test_partition_with_more_than_1024_blocks_bit_exact(gname, k):
    """Local search with more blocks than the compact CTA tables hold (1,024):
    the degree 513..8192 buckets use their full hashing-sized tables, and
    the split hubs accumulate by block without the per-part shared-memory
    pre-sum (more than 1,024 blocks)."""
    g = split_hub_graph(3) if gname == "split_hub" else gg.rmat(14, 8, 5)
    ref = O.partition(g, k, 0.03, seed=0)
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=0)
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)


@pytest.mark.parametrize("name,k", [("rmat16", 2), ("rgg", 8), ("weighted", 5), ("hub", 4),
                                    ("split_hub", 3)])
def test_partition_graph_driver_bit_exact(name, k):
    """The rounds run as one CUDA graph (device-side loop condition) give the
    same partition as the host-driven rounds and the oracle."""
    g = GRAPHS[name]()
    ref = O.partition(g, k, 0.03, seed=1)
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=1,
                                   cfg=P.default_config(graph_rounds=1))
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)
    assert res.stats["cluster_rounds"] == list(ref.stats.cluster_rounds[:len(res.stats["cluster_rounds"])])


def test_batch_graph_driver_equals_host_driver():
    graphs = [(gg.rmat(10 + i % 5, 8, 40 + i), [2, 4, 8, 16][i % 4]) for i in range(8)]
    graphs += [(gg.rgg2d(1500 + 900 * i, 60 + i), [2, 4, 8, 16][(i + 2) % 4]) for i in range(8)]
    items = [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), k=k, eps=0.03, seed=i)
             for i, (g, k) in enumerate(graphs)]
    a = P.sclap_partition_batch(items, device=True)
    b = P.sclap_partition_batch(items, device=True, cfg=P.default_config(graph_rounds=1))
    for x, y in zip(a, b):
        assert (x.status, x.cut) == (y.status, y.cut)
        assert np.array_equal(x.block.cpu().numpy(), y.block.cpu().numpy())


@pytest.mark.parametrize("name,k,size", [("rmat12", 2, 0), ("rgg", 4, 0), ("weighted", 16, 0),
                                         ("rmat16", 8, 3), ("hub", 64, 0)])
def test_partition_ensemble_bit_exact(name, k, size):
    """Ensemble clusterings during coarsening (configuration E)."""
    g = GRAPHS[name]()
    ref = O.partition(g, k, 0.03, seed=6, cfg=O.config(ensemble=1, ensemble_size=size))
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=6,
                                   cfg=P.default_config(ensemble=1, ensemble_size=size))
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)
    assert res.stats["level_n"] == list(ref.stats.level_n[:ref.stats.levels])


def test_batch_ensemble_mixed_sizes_equals_oracle():
    """Slots of one batch run ensembles of different sizes (l = 18, 7, 3)."""
    graphs = [(gg.rmat(11, 8, 70 + i), [2, 16, 64][i % 3]) for i in range(6)]
    items = [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), k=k, eps=0.03, seed=i)
             for i, (g, k) in enumerate(graphs)]
    out = P.sclap_partition_batch(items, device=True, cfg=P.default_config(ensemble=1))
    for i, ((g, k), r) in enumerate(zip(graphs, out)):
        ref = O.partition(g, k, 0.03, seed=i, cfg=O.config(ensemble=1))
        assert (r.status, r.cut) == (ref.status, ref.cut)
        assert np.array_equal(r.block.cpu().numpy(), ref.block)


@pytest.mark.parametrize("name,k,extra", [("rmat16", 2, {}), ("rgg", 8, {}), ("weighted", 5, {}),
                                          ("hub", 16, {}), ("rmat12", 4, {"ensemble": 1}),
                                          ("rgg", 3, {"cluster_active": 1})])
def test_partition_vcycles_bit_exact(name, k, extra):
    """Iterated V-cycles (configuration V, 3 cycles), alone and combined."""
    g = GRAPHS[name]()
    ref = O.partition(g, k, 0.03, seed=8, cfg=O.config(vcycles=3, **extra))
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=8,
                                   cfg=P.default_config(vcycles=3, **extra))
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)


def test_batch_vcycles_equals_oracle():
    graphs = [(gg.rmat(10 + i % 4, 8, 90 + i), [2, 4, 8, 16][i % 4]) for i in range(5)]
    graphs += [(gg.rgg2d(1200 + 800 * i, 95 + i), [2, 4, 8][i % 3]) for i in range(4)]
    items = [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), k=k, eps=0.03, seed=i)
             for i, (g, k) in enumerate(graphs)]
    out = P.sclap_partition_batch(items, device=True, cfg=P.default_config(vcycles=3))
    for i, ((g, k), r) in enumerate(zip(graphs, out)):
        ref = O.partition(g, k, 0.03, seed=i, cfg=O.config(vcycles=3))
        assert (r.status, r.cut) == (ref.status, ref.cut)
        assert np.array_equal(r.block.cpu().numpy(), ref.block)


def test_partition_host_api_and_seeds():
    g = gg.rmat(14, 8, 3)
    for seed in (0, 1, 2):
        ref = O.partition(g, 4, 0.05, seed=seed)
        res = P.sclap_partition(g.row_ptr, g.col, None, None, k=4, eps=0.05, seed=seed)
        assert res.cut == ref.cut and np.array_equal(res.block, ref.block)


@pytest.mark.parametrize("case", ["k1", "no_edges", "path", "tiny", "clique_ring", "eps0"])
def test_partition_edge_cases(case):
    if case == "k1":
        g, k, eps = gg.rmat(10, 8, 0), 1, 0.03
    elif case == "no_edges":
        g, k, eps = gg.from_edges(3000, [], []), 4, 0.03
    elif case == "path":
        g, k, eps = gg.path(5000), 2, 0.03
    elif case == "tiny":
        g, k, eps = gg.path(3), 3, 0.0
    elif case == "clique_ring":
        g, k, eps = gg.clique_ring(16, 50), 16, 0.03
    else:
        g, k, eps = gg.rgg2d(4000, 1), 8, 0.0
    ref = O.partition(g, k, eps, seed=4)
    res = P.sclap_partition_device(*dg(g), k=k, eps=eps, seed=4)
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)


def test_batch_equals_each_graph_alone():
    graphs = [(gg.rmat(10 + i % 4, 8, i), [2, 4, 8, 16][i % 4]) for i in range(6)]
    graphs += [(gg.rgg2d(1000 + 700 * i, i), [2, 4, 8, 16][(i + 1) % 4]) for i in range(6)]
    graphs.append((gg.random_weights(gg.rmat(11, 8, 9), 1), 5))
    items = [dict(row_ptr=g.row_ptr, col=g.col, node_w=g.node_w, edge_w=g.edge_w, k=k, eps=0.03,
                  seed=i) for i, (g, k) in enumerate(graphs)]
    res = P.sclap_partition_batch(items)
    dres = P.sclap_partition_batch(
        [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), node_w=dt(g.node_w), edge_w=dt(g.edge_w),
              k=k, eps=0.03, seed=i) for i, (g, k) in enumerate(graphs)], device=True)
    for i, (g, k) in enumerate(graphs):
        ref = O.partition(g, k, 0.03, seed=i)
        assert res[i].cut == ref.cut and np.array_equal(res[i].block, ref.block), i
        assert dres[i].cut == ref.cut
        assert np.array_equal(dres[i].block.cpu().numpy(), ref.block), i


def test_invalid_inputs_are_rejected():
    g = gg.rmat(8, 8, 0)
    bad = g.col.copy()
    bad[5] = g.n + 3                       # column out of range
    with pytest.raises(P.SclapError) as e:
        P.sclap_partition(g.row_ptr, bad, k=2)
    assert e.value.code == -2
    loop = g.col.copy()
    loop[g.row_ptr[7]] = 7 if g.row_ptr[8] > g.row_ptr[7] else loop[0]   # self-loop
    if g.row_ptr[8] > g.row_ptr[7]:
        with pytest.raises(P.SclapError):
            P.sclap_partition(g.row_ptr, loop, k=2)
    with pytest.raises(P.SclapError) as e:
        P.sclap_partition(g.row_ptr, g.col, k=g.n + 1)
    assert e.value.code == -1
    nw = np.ones(g.n, np.int32)
    nw[3] = 0                              # non-positive weight
    with pytest.raises(P.SclapError):
        P.sclap_partition(g.row_ptr, g.col, node_w=nw, k=2)
    # a failing call leaves the library usable
    ok = P.sclap_partition(g.row_ptr, g.col, k=2)
    assert ok.status == 0


def test_full_batch_sampled_against_oracle():
    # The benchmark's launch configuration: the whole 512-graph batch in one
    # device call; a sample of graphs (largest of each kind, a k = 16 one and
    # a few spread over the batch) is recomputed by the oracle one by one.
    import bench
    graphs = bench.workload(512, 0)
    items = [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), k=k, eps=eps, seed=0)
             for g, k, eps in graphs]
    res = P.sclap_partition_batch(items, device=True)
    assert all(r.status == 0 for r in res)
    sizes = [g.n for g, _, _ in graphs]
    rmat_big = max(range(0, 512, 2), key=lambda i: sizes[i])
    rgg_big = max(range(1, 512, 2), key=lambda i: sizes[i])
    k16 = next(i for i, (_, k, _) in enumerate(graphs) if k == 16)
    sample = sorted({rmat_big, rgg_big, k16, 0, 1, 255, 511})
    for i in sample:
        g, k, eps = graphs[i]
        ref = O.partition(g, k, eps, seed=0)
        assert res[i].cut == ref.cut, i
        assert np.array_equal(res[i].block.cpu().numpy(), ref.block), i
    # every graph balanced, cut equals a recount
    for i in range(0, 512, 37):
        g, k, eps = graphs[i]
        b = res[i].block.cpu().numpy()
        Lmax, _ = O.bounds(g.n, 1, k, eps)
        assert np.bincount(b, minlength=k).max() <= Lmax
        assert O.cut(g, b) == res[i].cut


def _heavy(g, seed, bits=22):
    """Edge weights up to 2^bits: the total arc weight is far above 2^32, so
    the propose tables must accumulate in 64 bits (coarse edges stay below
    2^31 for the inputs used here)."""
    h = gg.random_weights(g, seed, max_node_w=3, max_edge_w=1 << bits)
    assert int(h.edge_w.astype(np.int64).sum()) > (1 << 32)
    return h


@pytest.mark.parametrize("name,k", [("hub", 4), ("rmat12", 2), ("rmat16", 8)])
def test_heavy_edge_weights_bit_exact(name, k):
    g = _heavy(GRAPHS[name](), 17)
    ref = O.partition(g, k, 0.03, seed=4)
    res = P.sclap_partition_device(*dg(g), k=k, eps=0.03, seed=4)
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)


def test_batch_with_one_heavy_graph_equals_oracle():
    """One heavy graph puts the whole batch on 64-bit sums; the light graphs'
    results must not change."""
    gs = [(gg.rmat(12, 8, 31), 4), (_heavy(hub_graph(5), 3, bits=20), 2), (gg.rgg2d(3000, 32), 8),
          (gg.random_weights(gg.rmat(11, 8, 33), 34), 16)]
    items = [dict(row_ptr=dt(g.row_ptr), col=dt(g.col), node_w=dt(g.node_w), edge_w=dt(g.edge_w),
                  k=k, eps=0.03, seed=40 + i) for i, (g, k) in enumerate(gs)]
    res = P.sclap_partition_batch(items, device=True)
    for i, (g, k) in enumerate(gs):
        ref = O.partition(g, k, 0.03, seed=40 + i)
        assert (res[i].status, res[i].cut) == (ref.status, ref.cut), i
        assert np.array_equal(res[i].block.cpu().numpy(), ref.block), i


def test_coarse_edge_weight_overflow_reported_like_the_oracle():
    """Edge weights up to 2^22 around a degree-9000 hub: merged coarse edges
    pass 2^31.  The oracle stops with its overflow code; the device call
    fails with SCLAP_EOVERFLOW."""
    g = gg.random_weights(hub_graph(5), 3, max_node_w=3, max_edge_w=1 << 22)
    with pytest.raises(RuntimeError, match="rc=-2"):
        O.partition(g, 2, 0.03, seed=4)
    with pytest.raises(P.SclapError) as e:
        P.sclap_partition_device(*dg(g), k=2, eps=0.03, seed=4)
    assert e.value.code == P.EOVERFLOW


def test_scale19_rmat_bit_exact_both_drivers():
    """A larger input (R-MAT scale 19, 524,288 nodes): the whole partition
    bit-exact with the oracle under both round drivers; the reported cut
    equals an independent recount on the device."""
    g = gg.rmat(19, 8, 2)
    ref = O.partition(g, 16, 0.03, seed=3)
    rp, col = dt(g.row_ptr), dt(g.col)
    for gr in (0, 1):
        res = P.sclap_partition_device(rp, col, k=16, eps=0.03, seed=3,
                                       cfg=P.default_config(graph_rounds=gr))
        assert (res.status, res.cut) == (ref.status, ref.cut)
        assert np.array_equal(res.block.cpu().numpy(), ref.block)
        assert P.sclap_cut(rp, col, None, res.block) == res.cut


def test_large_single_graphs_bit_exact():
    """The large single-graph workload at full size, one graph per call as
    the benchmark runs it: R-MAT scale 22, edge factor 16 (4,194,304 nodes,
    ~128M arcs; generated on the device by graphgen.device), k = 8, seed 0;
    and a 2D RGG with 2^22 nodes, k = 64.  Blocks, cut and level sizes are
    bit-exact with the oracle (run in spawn-started worker processes), and
    the cut equals a device recount."""
    import multiprocessing as mp
    import _oracle_jobs as J
    from graphgen.device import rmat_torch

    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        rgg_job = pool.apply_async(J.rgg_and_partition, (1 << 22, 0, 64, 0.03, 0))
        rp, col = rmat_torch(22, 16, 0, device=DEV)
        hrp, hcol = rp.cpu().numpy(), col.cpu().numpy()
        assert hrp.size - 1 == 1 << 22 and hcol.size > 100_000_000
        rmat_job = pool.apply_async(J.partition, (hrp, hcol, 8, 0.03, 0))
        res = P.sclap_partition_device(rp, col, k=8, eps=0.03, seed=0)
        blk, cut, status, level_n = rmat_job.get()
        assert (res.status, res.cut) == (status, cut)
        assert np.array_equal(res.block.cpu().numpy(), blk)
        assert res.stats["level_n"] == level_n
        assert P.sclap_cut(rp, col, None, res.block) == res.cut
        del rp, col
        grp, gcol, blk, cut, status, level_n = rgg_job.get()
        trp, tcol = dt(grp), dt(gcol)
        res = P.sclap_partition_device(trp, tcol, k=64, eps=0.03, seed=0)
        assert (res.status, res.cut) == (status, cut)
        assert np.array_equal(res.block.cpu().numpy(), blk)
        assert res.stats["level_n"] == level_n
        assert P.sclap_cut(trp, tcol, None, res.block) == res.cut


@pytest.mark.parametrize("maker,k,trials,rounds", [
    (lambda: gg.rgg2d(300000, 6), 2, 1, 0),          # growing + water-filling alone
    (lambda: gg.rmat(19, 8, 7), 2, 2, 0),            # ~300k nodes with neighbours
    (lambda: gg.random_weights(gg.rgg2d(280000, 8), 9), 2, 2, 10),
    (lambda: gg.rgg2d(20000, 10), 16, 4, 10),        # small blocks: one CTA per trial
    (lambda: gg.rgg2d(60000, 11), 2, 3, 10),         # 30k nodes per block: groups
])
def test_initial_partition_of_few_large_trials_bit_exact(maker, k, trials, rounds):
    """Few trials with blocks of more than 2^14 nodes on average: each trial
    is grown by a group of CTAs (one cooperative launch) instead of one CTA;
    blocks, cut and best trial equal the oracle's (the last case stays on
    the one-CTA kernel)."""
    g = maker()
    cV = int(g.node_w.sum())
    Lmax, _ = O.bounds(cV, int(g.node_w.max()), k, 0.03)
    avg = -(-cV // k)
    cfg_o = O.config(ip_trials=trials, lp_rounds_refine=rounds)
    ob, ocut, obest = O.initial_partition(g, k, Lmax, avg, seed=12, level=1, cfg=cfg_o)
    tb, cut, best = P.sclap_initial_partition(
        *dg(g), k, Lmax, avg, 12, 1, cfg=P.default_config(ip_trials=trials, lp_rounds_refine=rounds))
    assert (cut, best) == (ocut, obest)
    assert np.array_equal(tb.cpu().numpy(), ob)

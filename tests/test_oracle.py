"""CPU pins for the oracle (no GPU).

Each test checks the oracle against something other than itself: published
generator outputs, closed forms, invariants stated in the paper, special cases
and brute force on tiny graphs.  Paper references are to Meyerhenke, Sanders,
Schulz, "Partitioning Complex Networks via Size-constrained Clustering".
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
M64 = 2**64 - 1


def recount_cut(g, block):
    """From-scratch cut: each undirected edge once (u < v), Sec. 2.1."""
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    once = src < g.col
    diff = block[src[once]] != block[g.col[once]]
    return int(g.edge_w[once][diff].sum())


def block_weights(g, block, k):
    return np.bincount(block, weights=g.node_w, minlength=k).astype(np.int64)


def brute_force_min_cut(g, Lmax):
    """Optimal balanced bisection by enumeration (node 0 fixed in block 0)."""
    n = g.n
    masks = np.arange(1 << (n - 1), dtype=np.int64) << 1  # bit v = block of v; v0 -> 0
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    once = src < g.col
    u, v, w = src[once], g.col[once], g.edge_w[once].astype(np.int64)
    cut = np.zeros(masks.size, np.int64)
    for a, b, ww in zip(u, v, w):
        cut += (((masks >> a) ^ (masks >> b)) & 1) * ww
    bits = (masks[:, None] >> np.arange(n)[None, :]) & 1
    w1 = (bits * g.node_w[None, :]).sum(1)
    w0 = int(g.node_w.sum()) - w1
    ok = (w0 <= Lmax) & (w1 <= Lmax)
    return int(cut[ok].min())


# ---------------------------------------------------------------- generator
def test_mix64_matches_published_splitmix64_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for i, hexv in rows:
        assert O.mix64((int(i) * GAMMA) & M64) == int(hexv, 16)


def test_hkey_is_a_chain_of_mix64():
    s, p, l, r = 7, 2, 3, 9
    assert O.hkey(s, p, l, r) == O.mix64(O.mix64(O.mix64(O.mix64(s) ^ p) ^ l) ^ r)


# ---------------------------------------------------------------- bounds
@pytest.mark.parametrize("cV,k,eps,L", [
    (65536, 2, 0.03, 33751),    # floor(1.03 * 32768)
    (100, 2, 0.03, 51),         # floor(1.03 * 50)
    (10, 3, 0.03, 4),           # floor(1.03 * ceil(10/3)=4)
    (1000, 4, 0.0, 250),        # eps = 0: perfect balance
    (7, 7, 0.5, 1),             # floor(1.5 * 1)
    (101, 2, 1.0, 102),         # floor(2 * 51)
])
def test_balance_bound_closed_form(cV, k, eps, L):
    # Sec. 2.1: for unit weights |V_i| <= (1+eps) * ceil(|V|/k).
    Lmax, U = O.bounds(cV, 1, k, eps, 18)
    assert Lmax == L
    # Sec. 3.1: U = max(max_v c(v), W) with W = Lmax / f.
    assert U == max(1, L // 18)


def test_cluster_bound_uses_heaviest_node():
    Lmax, U = O.bounds(1000, 500, 2, 0.03, 18)
    assert U == 500 and Lmax == 515


# ---------------------------------------------------------------- cut, balance
@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("k", [2, 3, 8])
def test_partition_cut_recount_and_balance(variant, k):
    for seed, g in enumerate([gg.rmat(10, 8, 1), gg.rgg2d(3000, 2),
                              gg.random_weights(gg.rmat(9, 6, 3), 5)]):
        r = O.partition(g, k, 0.03, seed, variant=variant)
        assert r.status == O.OK
        assert r.block.min() >= 0 and r.block.max() < k
        assert r.cut == recount_cut(g, r.block)
        bw = block_weights(g, r.block, k)
        Lmax, _ = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), k, 0.03)
        assert bw.max() <= Lmax and r.max_block_weight == bw.max()


def test_cut_function_against_recount():
    g = gg.random_weights(gg.gnp(60, 0.1, 4), 1)
    rng = np.random.default_rng(0)
    for _ in range(5):
        b = rng.integers(0, 5, g.n).astype(np.int32)
        assert O.cut(g, b) == recount_cut(g, b)


# ---------------------------------------------------------------- clustering
@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_cluster_weights_respect_U(variant):
    # Sec. 3.1: every cluster of a size-constrained clustering is <= U.
    for g, U in [(gg.rmat(11, 8, 2), 40), (gg.random_weights(gg.rgg2d(2000, 1), 3), 25),
                 (gg.star(300), 17)]:
        lab, rounds = O.cluster(g, U, seed=5, variant=variant)
        assert 1 <= rounds <= 10
        cw = np.bincount(lab, weights=g.node_w, minlength=g.n)
        assert cw.max() <= U
        # labels are ids of nodes (a cluster keeps its original representative id)
        assert lab.min() >= 0 and lab.max() < g.n


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_U_equal_one_gives_singletons(variant):
    # Sec. 2.1: with U = 1 on an unweighted graph the only feasible clustering
    # has every node on its own.
    g = gg.rmat(10, 8, 0)
    lab, _ = O.cluster(g, 1, seed=0, variant=variant)
    assert np.array_equal(lab, np.arange(g.n))
    # ... so contraction is the identity and coarsening stops at once.
    r = O.partition(g, 2, 0.03, 0, variant=variant, cfg=O.config(f=10**9, coarse_min_nodes=10))
    assert r.stats.levels == 1


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("k,s", [(4, 20), (8, 30), (16, 50)])
def test_clique_ring_clusters_are_the_cliques(variant, k, s):
    g = gg.clique_ring(k, s)
    lab, _ = O.cluster(g, s, seed=1, variant=variant)
    for q in range(k):
        assert len(set(lab[q * s:(q + 1) * s])) == 1
    assert len(set(lab)) == k


# ---------------------------------------------------------------- contraction
def _labelings(g, rng):
    yield rng.integers(0, max(1, g.n // 7), g.n).astype(np.int32)       # random clusters
    yield O.cluster(g, 30, seed=3)[0]                                    # LP clustering
    yield np.arange(g.n, dtype=np.int32)                                 # identity


def test_contraction_invariants():
    rng = np.random.default_rng(11)
    for g in [gg.random_weights(gg.rmat(10, 8, 4), 2), gg.rgg2d(1500, 5), gg.path(50)]:
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        for lab in _labelings(g, rng):
            c = O.contract(g, lab)
            cg = gg.Graph(c.row_ptr, c.col, c.node_w, c.edge_w)
            gg.validate(cg)                                  # canonical, symmetric
            # node weight of a cluster = sum of its members (Sec. 3.1)
            assert c.node_w.sum() == g.node_w.sum()
            used = np.unique(lab)
            assert c.n == used.size
            assert np.array_equal(c.cmap, np.searchsorted(used, lab))
            assert np.array_equal(c.node_w, np.bincount(c.cmap, weights=g.node_w).astype(np.int32))
            # coarse edge weight = fine weight minus the intra-cluster part
            intra = g.edge_w[lab[src] == lab[g.col]].sum()
            assert c.edge_w.sum() == g.edge_w.sum() - intra
            # a coarse partition and its projection have the same cut (Sec. 3.1)
            for kk in (2, 5):
                cb = rng.integers(0, kk, c.n).astype(np.int32)
                assert O.cut(cg, cb) == recount_cut(g, cb[c.cmap])
            # rows sorted by neighbour id
            for a in range(min(c.n, 200)):
                row = c.col[c.row_ptr[a]:c.row_ptr[a + 1]]
                assert np.all(np.diff(row) > 0)


def test_contraction_of_clique_ring():
    k, s = 6, 10
    g = gg.clique_ring(k, s)
    lab = (np.arange(g.n) // s * s).astype(np.int32)
    c = O.contract(g, lab)
    assert c.n == k and np.all(c.node_w == s)
    # a ring of k nodes with unit edges
    assert np.all(np.diff(c.row_ptr) == 2) and np.all(c.edge_w == 1)


# ---------------------------------------------------------------- special cases
@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_k_equals_one(variant):
    g = gg.rmat(10, 8, 2)
    r = O.partition(g, 1, 0.03, 0, variant=variant)
    assert np.all(r.block == 0) and r.cut == 0 and r.max_block_weight == g.n


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_empty_edge_set(variant):
    n, k = 1000, 4
    g = gg.from_edges(n, [], [])
    r = O.partition(g, k, 0.03, 0, variant=variant)
    assert r.cut == 0
    assert block_weights(g, r.block, k).max() <= O.bounds(n, 1, k, 0.03)[0]


def test_invalid_arguments_rejected():
    g = gg.path(10)
    with pytest.raises(RuntimeError):
        O.partition(g, 11, 0.03, 0)
    with pytest.raises(RuntimeError):
        O.partition(g, 0, 0.03, 0)
    with pytest.raises(RuntimeError):
        O.partition(g, 2, -0.1, 0)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("n", [20, 100, 1001, 5000])
def test_path_bisection_is_optimal(variant, n):
    # P_n, k = 2: the optimum cuts a single edge.
    for seed in range(2):
        assert O.partition(gg.path(n), 2, 0.03, seed, variant=variant).cut == 1


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("k,s", [(4, 20), (8, 30), (16, 50)])
def test_clique_ring_partition_cuts_only_ring_edges(variant, k, s):
    # k cliques joined in a ring, k blocks of size s: optimum = k ring edges;
    # as a path of cliques: k - 1.
    assert O.partition(gg.clique_ring(k, s), k, 0.03, 0, variant=variant).cut == k
    assert O.partition(gg.clique_ring(k, s, ring=False), k, 0.03, 0, variant=variant).cut == k - 1


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("r,c", [(10, 10), (20, 10), (40, 20)])
def test_grid_bisection_bounds(variant, r, c):
    # r x c grid (c <= r), k = 2: the optimum is c.  LP local search leaves
    # staircase boundaries, so only the lower bound is exact; the upper bound
    # records the quality observed for this heuristic.
    cut = O.partition(gg.grid(r, c), 2, 0.03, 0, variant=variant).cut
    assert c <= cut <= 2 * c


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_never_below_brute_force_optimum(variant):
    gaps = []
    for seed in range(12):
        n = 10 + seed % 7
        g = gg.gnp(n, 0.35, seed)
        if seed % 3 == 0:
            g = gg.random_weights(g, seed, max_node_w=3, max_edge_w=5)
        cV = int(g.node_w.sum())
        Lmax, _ = O.bounds(cV, int(g.node_w.max()), 2, 0.03)
        opt = brute_force_min_cut(g, Lmax)
        r = O.partition(g, 2, 0.03, seed, variant=variant)
        if r.status == O.OK:
            assert r.cut >= opt
            gaps.append(r.cut - opt)
    assert gaps and np.mean(gaps) <= 2.0


def test_brute_force_structured_cases_hit_the_optimum():
    for g in [gg.path(16), gg.clique_ring(2, 8, ring=False), gg.star(12)]:
        Lmax, _ = O.bounds(g.n, 1, 2, 0.03)
        opt = brute_force_min_cut(g, Lmax)
        for variant in (O.SYNC, O.SEQ):
            assert O.partition(g, 2, 0.03, 0, variant=variant).cut == opt


# ---------------------------------------------------------------- one LP round
def _conn_table(g, label, nlabels):
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    T = np.zeros((g.n, nlabels), np.int64)
    np.add.at(T, (src, label[g.col]), g.edge_w)
    return T


@pytest.mark.parametrize("mode", [O.MODE_CLUSTER, O.MODE_REFINE])
def test_single_colour_round_moves_are_strongest_eligible(mode):
    # With one colour class every node decides against the round-start state,
    # so each admitted move must go to a label of maximum connection among the
    # eligible ones, strictly better than staying (Sec. 3.1).
    rng = np.random.default_rng(3)
    g = gg.random_weights(gg.rmat(9, 8, 7), 2)
    if mode == O.MODE_CLUSTER:
        nl = g.n
        label = rng.integers(0, g.n // 4, g.n).astype(np.int32)
    else:
        nl = 6
        label = rng.integers(0, nl, g.n).astype(np.int32)
    W = np.bincount(label, weights=g.node_w, minlength=nl).astype(np.int64)
    bound = int(W.max()) + (3 if mode == O.MODE_CLUSTER else 20)
    T = _conn_table(g, label, nl)
    lab2, W2, moved, _ = O.lp_round(g, mode, label, W, bound, rkey=99, sub_rounds=1)
    assert moved == int((lab2 != label).sum()) and moved > 0
    assert W2.max() <= bound
    assert np.array_equal(W2, np.bincount(lab2, weights=g.node_w, minlength=nl))
    for v in np.nonzero(lab2 != label)[0]:
        cv = g.node_w[v]
        own = label[v]
        elig = (W + cv <= bound)
        elig[own] = False
        adjl = T[v] > 0
        best = T[v][elig & adjl].max()
        assert T[v, lab2[v]] == best and best > T[v, own]
        assert W[lab2[v]] + cv <= bound


def test_round_admission_never_overfills_a_target():
    # A star: every leaf proposes the hub's cluster; only U - 1 fit.
    g = gg.star(500)
    label = np.arange(g.n, dtype=np.int32)
    W = np.ones(g.n, np.int64)
    for S in (1, 3, 8):
        lab2, W2, moved, _ = O.lp_round(g, O.MODE_CLUSTER, label, W, 17, rkey=5, sub_rounds=S)
        assert W2.max() <= 17
        # the hub itself moves to one leaf in its colour class; leaves fill the hub cluster
        assert np.bincount(lab2, minlength=g.n)[0] >= 15


def test_overloaded_block_sheds_its_excess_only():
    # Local search with an overloaded block: its nodes must leave it (Sec. 3.1),
    # and the source-side cap stops departures once the excess is gone, so
    # with unit weights the block never drops below Lmax (target-side
    # competition may still reject some of its moves).
    g = gg.rgg2d(3000, 4)
    k = 4
    label = (np.arange(g.n) % k).astype(np.int32)
    label[np.nonzero(label != 0)[0][:60]] = 0
    W = np.bincount(label, minlength=k).astype(np.int64)
    Lmax = O.bounds(g.n, 1, k, 0.03)[0]
    assert W[0] > Lmax and (Lmax - W[1:]).sum() > W[0] - Lmax
    lab2, W2, moved, _ = O.lp_round(g, O.MODE_REFINE, label, W, Lmax, rkey=3, sub_rounds=1)
    assert Lmax <= W2[0] < W[0] and W[0] - W2[0] >= (W[0] - Lmax) // 2
    assert W2[1:].max() <= Lmax
    assert np.array_equal(W2, np.bincount(lab2, minlength=k))


def test_active_next_marks_neighbours_of_moved_nodes():
    g = gg.rmat(9, 8, 1)
    label = np.arange(g.n, dtype=np.int32)
    W = np.ones(g.n, np.int64)
    lab2, _, _, an = O.lp_round(g, O.MODE_CLUSTER, label, W, 8, rkey=1, sub_rounds=4,
                                want_next=True)
    moved = np.nonzero(lab2 != label)[0]
    expect = np.zeros(g.n, bool)
    for v in moved:
        expect[g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = True
    assert np.array_equal(an.astype(bool), expect)


# ---------------------------------------------------------------- growing, IP
def test_ggg_assigns_every_node_and_respects_target():
    for g in [gg.rmat(10, 8, 3), gg.random_weights(gg.rgg2d(2000, 3), 4)]:
        k = 5
        cV = int(g.node_w.sum())
        avg = -(-cV // k)
        blk, W = O.ggg(g, k, avg, tkey=12345)
        assert blk.min() >= 0 and blk.max() < k
        assert np.array_equal(W, np.bincount(blk, weights=g.node_w, minlength=k))
        assert W.sum() == cV
        # water-filling only tops up blocks below the fill level, so no block
        # exceeds avg by more than one node's weight
        assert W.max() <= avg + g.node_w.max()


def test_initial_partition_keeps_best_trial():
    g = gg.rgg2d(800, 9)
    k, cV = 4, 800
    Lmax, _ = O.bounds(cV, 1, k, 0.03)
    avg = cV // k
    blk, cut, best = O.initial_partition(g, k, Lmax, avg, seed=4, cfg=O.config(ip_trials=8))
    assert cut == recount_cut(g, blk)
    one, cut1, _ = O.initial_partition(g, k, Lmax, avg, seed=4, cfg=O.config(ip_trials=1))
    assert cut <= cut1
    assert 0 <= best < 8


def test_repair_restores_balance():
    g = gg.rmat(10, 8, 5)
    k = 4
    Lmax, _ = O.bounds(g.n, 1, k, 0.03)
    blk = np.zeros(g.n, np.int32)
    blk[g.n // 2:] = np.arange(g.n - g.n // 2) % 3 + 1
    blk2, rounds, rc = O.repair(g, k, Lmax, blk, seed=1)
    assert rc == O.OK and rounds >= 1
    assert block_weights(g, blk2, k).max() <= Lmax


# ---------------------------------------------------------------- determinism, quality
def test_deterministic_and_seed_dependent():
    g = gg.rmat(11, 8, 6)
    a = O.partition(g, 4, 0.03, 1)
    b = O.partition(g, 4, 0.03, 1)
    c = O.partition(g, 4, 0.03, 2)
    assert np.array_equal(a.block, b.block) and a.cut == b.cut
    assert not np.array_equal(a.block, c.block)


@pytest.mark.slow
def test_sync_mean_cut_within_5_percent_of_sequential():
    # Quality relation (not equality): the round-synchronous variant that the
    # GPU follows must stay within 5% of the paper's sequential SCLaP in mean
    # final cut over seeds 0-4 on the scale-16 R-MAT, k = 2.
    g = gg.rmat(16, 8, 0)
    seq = np.mean([O.partition(g, 2, 0.03, s, variant=O.SEQ).cut for s in range(5)])
    syn = np.mean([O.partition(g, 2, 0.03, s, variant=O.SYNC).cut for s in range(5)])
    assert syn <= 1.05 * seq


# ---------------------------------------------------------------- active nodes
# Active nodes during coarsening (Sec. 4 "Active Nodes"; configuration A of
# Table 2): in the first round every node is active, afterwards a node is
# active iff one of its neighbours changed its cluster in the previous round.

@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_active_coarsening_single_round_equals_plain(variant):
    g = gg.rmat(11, 8, 5)
    one = dict(lp_rounds_coarse=1)
    a, _ = O.cluster(g, 40, 3, variant=variant, cfg=O.config(cluster_active=1, **one))
    b, _ = O.cluster(g, 40, 3, variant=variant, cfg=O.config(cluster_active=0, **one))
    assert np.array_equal(a, b)


def test_active_coarsening_follows_the_definition():
    """orc_cluster with active nodes equals rounds driven from Python, where
    each round's active set is recomputed from the definition: the
    neighbours of the nodes whose label changed in the round before."""
    g = gg.rgg2d(1500, 7)
    U, seed, level = 25, 11, 2
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    label = np.arange(g.n, dtype=np.int32)
    W = g.node_w.astype(np.int64)
    active = np.ones(g.n, dtype=np.uint8)
    for R in range(1, 6):
        rkey = O.hkey(seed, O.PH_CLUSTER, level, R - 1)
        new, W, moved, _ = O.lp_round(g, O.MODE_CLUSTER, label, W, U, rkey, 8, active_cur=active)
        changed = new != label
        active = np.zeros(g.n, dtype=np.uint8)
        active[g.col[changed[src]]] = 1
        label = new
        got, rounds = O.cluster(g, U, seed, level=level,
                                cfg=O.config(cluster_active=1, lp_rounds_coarse=R))
        if rounds < R:          # stopped early by the 5% rule: nothing more to compare
            break
        assert np.array_equal(got, label), R


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_active_coarsening_respects_U(variant):
    g = gg.random_weights(gg.rmat(12, 8, 2), 4, max_node_w=5)
    U = 60
    lab, _ = O.cluster(g, U, 1, variant=variant, cfg=O.config(cluster_active=1))
    assert np.bincount(lab, weights=g.node_w, minlength=g.n).max() <= U


@pytest.mark.parametrize("active", [0, 1])
def test_random_order_recovers_cliques(active):
    """Configuration R (random node order, sequential variant): cliques joined
    by single edges are still found exactly when U equals the clique size."""
    k, s = 6, 7
    g = gg.clique_ring(k, s)
    lab, _ = O.cluster(g, s, 4, variant=O.SEQ,
                       cfg=O.config(random_order=1, cluster_active=active))
    groups = {tuple(np.flatnonzero(lab == c)) for c in np.unique(lab)}
    assert groups == {tuple(range(q * s, (q + 1) * s)) for q in range(k)}


# ------------------------------------------------------ clustering hierarchy
# Clustering without a partitioning target (Sec. 3.1 clustering and
# contraction, repeated as in the coarsening phase).

def _hierarchy_by_hand(g, U, stop, seed, cfg):
    """The repetition written out: cluster, contract, keep the contraction
    only if it removes >= 5% of the nodes, compose the maps."""
    comm = np.arange(g.n)
    sizes = [g.n]
    cur, level = g, 0
    while cur.n > stop and level + 1 < cfg.max_levels:
        lab, _ = O.cluster(cur, U, seed, level=level, cfg=cfg)
        c = O.contract(cur, lab)
        if 20 * (cur.n - c.n) < cur.n:
            break
        comm = c.cmap[comm]
        cur = gg.Graph(c.row_ptr, c.col, c.node_w, c.edge_w)
        level += 1
        sizes.append(cur.n)
    return comm, level, sizes


@pytest.mark.parametrize("maker", [lambda: gg.rmat(12, 8, 3), lambda: gg.rgg2d(3000, 2),
                                   lambda: gg.random_weights(gg.rmat(11, 8, 1), 2)])
def test_cluster_hierarchy_is_repeated_cluster_and_contract(maker):
    g = maker()
    cfg = O.config()
    for U, stop in ((30, 100), (200, 1)):
        comm, levels, sizes = O.cluster_hierarchy(g, U, stop, 9, cfg=cfg)
        ref = _hierarchy_by_hand(g, U, stop, 9, cfg)
        assert levels == ref[1] and sizes == ref[2]
        assert np.array_equal(comm, ref[0])
        # every community is a coarse node: at most U in weight
        assert np.bincount(comm, weights=g.node_w).max() <= U


def test_cluster_hierarchy_special_cases():
    g = gg.rmat(10, 8, 2)
    comm, levels, sizes = O.cluster_hierarchy(g, 1, 1, 0)      # U = 1: nothing merges
    assert levels == 0 and sizes == [g.n] and np.array_equal(comm, np.arange(g.n))
    comm, levels, _ = O.cluster_hierarchy(g, 50, g.n, 0)       # already small enough
    assert levels == 0 and np.array_equal(comm, np.arange(g.n))
    # cliques of size s joined in a ring, U = s: one contraction finds the
    # cliques, after which no cluster can grow and the hierarchy stops
    k, s = 12, 9
    g = gg.clique_ring(k, s)
    comm, levels, sizes = O.cluster_hierarchy(g, s, 1, 5)
    assert levels == 1 and sizes == [k * s, k]
    for q in range(k):
        assert len(set(comm[q * s:(q + 1) * s])) == 1
    assert len(set(comm)) == k


# ----------------------------------------------------- ensemble clusterings
# Sec. 4 "Ensemble Clusterings" (configuration E): the overlay puts two nodes
# together iff every input clustering does; each coarsening level contracts
# the overlay of l clusterings (Sec. 5: l = 18 / 7 / 3 by k).

def test_overlay_is_the_intersection_brute_force():
    rng = np.random.default_rng(3)
    for n, ka, kb in [(12, 3, 4), (30, 5, 2), (25, 25, 1)]:
        a = rng.integers(0, ka, n).astype(np.int32) * 7 + 100     # arbitrary ids
        b = rng.integers(0, kb, n).astype(np.int32) * 3
        o = O.overlay(a, b)
        for u in range(n):
            for v in range(n):
                assert (o[u] == o[v]) == (a[u] == a[v] and b[u] == b[v])
        # numbered 0, 1, ... by first occurrence in node order
        firsts = [o[v] for v in range(n) if o[v] not in set(o[:v])]
        assert firsts == list(range(len(firsts)))


def test_overlay_of_ensemble_refines_each_clustering_and_keeps_U():
    g = gg.rmat(11, 8, 6)
    U = 40
    labs = [O.cluster(g, U, seed=100 + j)[0] for j in range(4)]
    o = labs[0]
    for lab in labs[1:]:
        o = O.overlay(o, lab)
    assert len(np.unique(o)) >= max(len(np.unique(l)) for l in labs)
    assert np.bincount(o, weights=g.node_w).max() <= U


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_ensemble_of_one_is_plain_coarsening(variant):
    g = gg.rmat(13, 8, 2)
    a = O.partition(g, 4, 0.03, seed=3, variant=variant, cfg=O.config(ensemble=1, ensemble_size=1))
    b = O.partition(g, 4, 0.03, seed=3, variant=variant)
    assert a.cut == b.cut and np.array_equal(a.block, b.block)


@pytest.mark.parametrize("k", [2, 16, 64])
def test_ensemble_partition_is_balanced_and_counted(k):
    g = gg.rgg2d(6000, 4)
    r = O.partition(g, k, 0.03, seed=1, cfg=O.config(ensemble=1, ensemble_size=3))
    Lmax, _ = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), k, 0.03)
    assert np.bincount(r.block, minlength=k).max() <= Lmax
    assert r.cut == O.cut(g, r.block)


# ------------------------------------------------------------- V-cycles
# Iterated V-cycles (Sec. 4 "Iterated Multilevel Algorithms", App. A): later
# cycles coarsen with clusterings inside the blocks of the current partition,
# start from it on the coarsest graph and refine on the way back.

def _restricted_clusters_ok(g, lab, blk):
    """Every cluster lies inside one block."""
    for c in np.unique(lab):
        if len(np.unique(blk[lab == c])) != 1:
            return False
    return True


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_vcycles_one_equals_plain(variant):
    g = gg.rmat(12, 8, 3)
    a = O.partition(g, 4, 0.03, seed=2, variant=variant, cfg=O.config(vcycles=1))
    b = O.partition(g, 4, 0.03, seed=2, variant=variant)
    assert a.cut == b.cut and np.array_equal(a.block, b.block)


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
def test_clustering_in_blocks(variant):
    g = gg.rmat(12, 8, 4)
    U = 50
    blk = np.random.default_rng(1).integers(0, 3, g.n).astype(np.int32)
    lab, _ = O.cluster_in_blocks(g, U, 5, blk, variant=variant)
    assert _restricted_clusters_ok(g, lab, blk)
    assert np.bincount(lab, weights=g.node_w, minlength=g.n).max() <= U
    # one block for everybody: plain clustering
    same, _ = O.cluster_in_blocks(g, U, 5, np.zeros(g.n, np.int32), variant=variant)
    assert np.array_equal(same, O.cluster(g, U, 5, variant=variant)[0])
    # a block per node: nothing can merge
    alone, _ = O.cluster_in_blocks(g, U, 5, np.arange(g.n, dtype=np.int32), variant=variant)
    assert np.array_equal(alone, np.arange(g.n))


@pytest.mark.parametrize("variant", [O.SYNC, O.SEQ])
@pytest.mark.parametrize("maker,k", [(lambda: gg.rmat(13, 8, 5), 2), (lambda: gg.rgg2d(8000, 3), 8),
                                     (lambda: gg.random_weights(gg.rmat(12, 8, 1), 2), 4)])
def test_vcycles_never_worsen_a_balanced_cut(variant, maker, k):
    """A respecting clustering contracts no cut edge, so a cycle starts from
    the previous cut; sequential refinement of a balanced partition makes
    only positive-gain moves, so the cut can only drop (App. A).  In the
    synchronous variant two adjacent nodes of one colour class may move
    together, so there it is a property of these instances, not a theorem."""
    g = maker()
    Lmax, _ = O.bounds(int(g.node_w.sum()), int(g.node_w.max()), k, 0.03)
    prev = None
    for V in (1, 2, 3):
        r = O.partition(g, k, 0.03, seed=7, variant=variant, cfg=O.config(vcycles=V))
        assert r.cut == O.cut(g, r.block)
        assert np.bincount(r.block, weights=g.node_w, minlength=k).max() <= Lmax
        if prev is not None:
            assert r.cut <= prev
        prev = r.cut


# ------------------------------------------- admission order (hand-computed)
# One synchronous sub-round (S = 1), target side: when the proposals into a
# cluster do not all fit, the longest prefix in (larger gain, smaller
# priority hash, smaller node id) order whose weight fits is admitted, and
# admission stops at the first proposal that does not fit (Sec. 3.1 "will
# not become overloaded", read for simultaneous moves).  The expected sets
# below are worked out by hand; the comments name the plausible mistakes
# each case rejects.

def _admission_graph(room):
    """Target cluster 0 = {t=0, a=1} (edge t-a of weight 100 keeps both at
    home).  Proposers p = 2..6, each with a partner q = p + 5 in its own
    cluster (label p); edge p-t of weight w, edge p-q of weight o.  Gains
    w - o and node weights c(p):
        p : 2  3  4  5  6
        w : 10 12  8  6  3     (connection to cluster 0)
        o :  1  8  1  1  1     (connection to its own cluster)
      gain:  9  4  7  5  2
      c(p):  2  1  3  1  1
    Cluster 0 weighs 2; U = 2 + room."""
    w = {2: 10, 3: 12, 4: 8, 5: 6, 6: 3}
    o = {2: 1, 3: 8, 4: 1, 5: 1, 6: 1}
    cp = {2: 2, 3: 1, 4: 3, 5: 1, 6: 1}
    s, d, ww = [0], [1], [100]
    for p in range(2, 7):
        s += [p, p]
        d += [0, p + 5]
        ww += [w[p], o[p]]
    g = gg.from_edges(12, s, d, w=ww)
    for p in range(2, 7):
        g.node_w[p] = cp[p]
    label = np.array([0, 0, 2, 3, 4, 5, 6, 2, 3, 4, 5, 6], np.int32)
    W = np.bincount(label, weights=g.node_w, minlength=12).astype(np.int64)
    return g, label, W, int(W[0]) + room


@pytest.mark.parametrize("room,admitted", [
    # gain order 2 (c 2), 4 (c 3), 5, 3, 6 (c 1 each):
    (4, {2}),          # 2 fits (2), 4 does not (5 > 4): stop.  Skipping instead
                       # would also admit 5 and 3; ordering by connection (3, 2, 4)
                       # admits {3, 2}; ascending gain admits {6, 3, 5}
    (5, {2, 4}),       # 2 + 3 = 5 fits, then 5 would make 6
    (7, {2, 4, 5, 3}),  # 6 would make 8
    (8, {2, 3, 4, 5, 6}),  # everything fits: all admitted
    (1, {5}),          # a move that would overload cluster 0 by itself is not
                       # eligible (2 and 4 do not propose); of 5, 3, 6 (c 1 each)
                       # the largest gain, 5, takes the one unit
])
def test_admission_admits_the_longest_prefix_in_gain_order(room, admitted):
    g, label, W, U = _admission_graph(room)
    lab2, W2, moved, _ = O.lp_round(g, O.MODE_CLUSTER, label, W, U, rkey=12345, sub_rounds=1)
    got = {int(v) for v in np.nonzero(lab2 != label)[0]}
    # every proposer that does not fit in cluster 0 stays (its only other
    # option, staying, is what a rejected proposal means)
    assert got == admitted
    assert all(lab2[v] == 0 for v in got)
    assert moved == len(admitted) and W2[0] == W[0] + sum(int(g.node_w[v]) for v in admitted)
    assert W2[0] <= U


def test_admission_ties_in_gain_go_to_the_smaller_priority_hash():
    """Two proposers (nodes 2, 3) of equal gain and weight into cluster 0,
    room for one.  The priority is the low 32 bits of the node's round hash
    mix64(rkey ^ v) (mix64 is pinned to the published SplitMix64 outputs);
    the smaller one wins.  Round keys are chosen so that each node wins in
    one of them: ordering by node id, by descending hash or by the high hash
    bits fails one of the two."""
    s, d, ww = [0, 2, 3], [1, 0, 0], [100, 5, 5]
    g = gg.from_edges(4, s, d, w=ww)
    label = np.array([0, 0, 2, 3], np.int32)
    W = np.bincount(label, weights=g.node_w, minlength=4).astype(np.int64)
    U = int(W[0]) + 1

    def prio(rkey, v):
        return O.mix64(rkey ^ v) & 0xFFFFFFFF

    def hi(rkey, v):
        return O.mix64(rkey ^ v) >> 32

    seen = set()
    for rkey in range(1, 400):
        win = 2 if prio(rkey, 2) < prio(rkey, 3) else 3
        # keep only keys where the high half would pick the other node, so a
        # high-bits mistake is caught as well
        if (hi(rkey, 2) < hi(rkey, 3)) == (win == 2):
            continue
        if win in seen:
            continue
        seen.add(win)
        lab2, _, moved, _ = O.lp_round(g, O.MODE_CLUSTER, label, W, U, rkey=rkey, sub_rounds=1)
        assert moved == 1 and lab2[win] == 0 and lab2[5 - win] == 5 - win, rkey
        if seen == {2, 3}:
            break
    assert seen == {2, 3}


# ------------------------------------------------- greedy growing (by hand)
# Greedy graph growing as the initial partitioning reads it (the paper
# leaves KaHIP's initial partitioner unspecified): block j starts at the
# unassigned node with neighbours of smallest seed hash; every step absorbs,
# in increasing id order, the unassigned nodes adjacent to the block while
# its weight stays <= ceil(c(V)/k), stopping at the first that would
# overflow; leftovers are water-filled into the lightest blocks.

def _ggg_tkey(g, k, want, level=0):
    """A trial key whose block seeds are the nodes `want` (block j grows from
    want[j]); seeds are the smallest mix64(hkey(tkey, GGG, level, j) ^ v)
    over the nodes not yet taken.  Searched, not assumed."""
    nonisolated = [v for v in range(g.n) if g.row_ptr[v + 1] > g.row_ptr[v]]
    for tkey in range(1, 20000):
        taken = set()
        ok = True
        for j, seed in enumerate(want):
            skey = O.hkey(tkey, O.PH_GGG, level, j)
            cand = [v for v in nonisolated if v not in taken]
            best = min(cand, key=lambda v: O.mix64(skey ^ v))
            if best != seed:
                ok = False
                break
            # the rest of block j is not known here; it is enough that the
            # seed of block j+1 lies outside block j (true for the cases below)
            taken.add(best)
        if ok:
            return tkey
    raise AssertionError("no trial key found")


def test_ggg_grows_by_adjacency_steps_in_id_order():
    """Path 0-1-...-10, unit weights, k = 2, avg = ceil(11/2) = 6.
    Block 0 from node 5: step 1 takes {4, 6} (weight 3), step 2 {3, 7} (5),
    step 3 meets candidates 2 and 8 in id order: 2 fits (6), 8 does not
    -> block 0 = {2..7}.  Block 1 from node 10: {9}, then {8}, then no
    unassigned neighbour -> {8, 9, 10} (weight 3).  Leftovers 0 and 1
    (weight 2) are water-filled: level 5 frees 2 units in block 1 only.
    Absorbing in descending id order would take 8 instead of 2; growing
    without adjacency would start with 0, 1, 2."""
    g = gg.path(11)
    tkey = _ggg_tkey(g, 2, [5, 10])
    blk, W = O.ggg(g, 2, 6, tkey)
    assert blk.tolist() == [1, 1, 0, 0, 0, 0, 0, 0, 1, 1, 1]
    assert W.tolist() == [6, 5]


def test_ggg_stops_at_the_first_node_that_would_overflow():
    """Paths 0-1-2-3 and 4-5-6-7-8 joined by the edge 2-5; c(3) = 6, every
    other node weighs 1: c(V) = 14, k = 2, avg = 7.
    Block 0 from node 2: candidates 1, 3, 5 in id order; 1 fits (2), 3 would
    make 8 -> stop (5 is not taken although it would fit).  Step 2: 0 fits
    (3), 3 would overflow -> stop.  Step 3: only 3 is adjacent and does not
    fit -> block 0 = {0, 1, 2} (weight 3).
    Block 1 from node 8 walks 7, 6, 5, 4 (weight 5); 3 is not adjacent.
    Leftover 3 (weight 6) goes to the lightest block, 0: W = [9, 5].
    Skipping the overflowing node instead of stopping would give block 0
    = {0, 1, 2, 4, 5, 6, 7}."""
    s = [0, 1, 2, 4, 5, 6, 7, 2]
    d = [1, 2, 3, 5, 6, 7, 8, 5]
    g = gg.from_edges(9, s, d)
    g.node_w[3] = 6
    tkey = _ggg_tkey(g, 2, [2, 8])
    blk, W = O.ggg(g, 2, 7, tkey)
    assert blk.tolist() == [0, 0, 0, 0, 1, 1, 1, 1, 1]
    assert W.tolist() == [9, 5]


# ------------------------------------------- sequential node order (by hand)
def test_sequential_round_visits_nodes_in_increasing_degree_order():
    """Sec. 4 "Node Ordering": the sequential algorithm visits nodes in
    increasing degree (equal degrees in the round's hash order, ascending).
    Path 0-1-2 with w(0,1) = 5, w(1,2) = 3, unit node weights, U = 2, one
    round.  Degrees 1, 2, 1: node 1 comes last, 0 and 2 in hash order.
      2 first: 2 joins 1's cluster (full now); 0 cannot; 1 then prefers
               cluster 0 (5 > 3) and moves there -> [0, 0, 1].
      0 first: 0 joins 1's cluster; 2 cannot; 1 stays (5 > 3) -> [1, 1, 2].
    Id order (0, 1, 2) gives [1, 1, 2] for every seed; decreasing degree
    (1 first) gives [0, 0, 2]."""
    g = gg.from_edges(3, [0, 1], [1, 2], w=[5, 3])
    cfg = O.config(lp_rounds_coarse=1)
    outcomes = set()
    for seed in range(64):
        rk = O.hkey(seed, O.PH_CLUSTER, 0, 0)
        two_first = O.mix64(rk ^ 2) < O.mix64(rk ^ 0)
        lab, rounds = O.cluster(g, 2, seed, variant=O.SEQ, cfg=cfg)
        assert rounds == 1
        assert lab.tolist() == ([0, 0, 1] if two_first else [1, 1, 2]), seed
        outcomes.add(two_first)
    assert outcomes == {True, False}

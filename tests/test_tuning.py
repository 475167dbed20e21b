"""Launch tuning (sclap_set_tuning / sclap_autotune): the setting changes how
the LP sweep is scheduled and never what it computes.

The CPU tests check the setting's validation; the GPU tests partition the
same batch under settings that move every degree bucket between kernels,
grid sizes and stream layouts, and require the oracle's result every time.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_1402_3281_gb300 as P

DEFAULT = dict(small_max_deg=16, small_ctas_per_sm=8, warp_ctas_per_sm=8, admit_ctas_per_sm=16,
               concurrent=1, pdl=1, fused_admission=0, contract_table_slots=0, ip_trial_group=0,
               contract_merge=0)


@pytest.fixture
def restore_tuning():
    before = P.get_tuning().to_dict()
    yield
    P.set_tuning(**before)


def test_default_tuning(restore_tuning):
    P.set_tuning(**DEFAULT)
    assert P.get_tuning().to_dict() == DEFAULT


@pytest.mark.parametrize("field,bad", [("small_max_deg", 12), ("small_max_deg", 32),
                                       ("small_ctas_per_sm", 0), ("warp_ctas_per_sm", 33),
                                       ("admit_ctas_per_sm", 65), ("concurrent", 2),
                                       ("concurrent", -1), ("pdl", 2),
                                       ("fused_admission", 2), ("fused_admission", -1),
                                       ("contract_table_slots", -5), ("ip_trial_group", -1),
                                       ("contract_merge", 2), ("contract_merge", -1)])
def test_out_of_range_values_are_rejected_and_leave_the_setting(restore_tuning, field, bad):
    P.set_tuning(**DEFAULT)
    with pytest.raises(P.SclapError) as e:
        P.set_tuning(**{field: bad})
    assert e.value.code == P.EINVAL
    assert P.get_tuning().to_dict() == DEFAULT


def test_set_tuning_round_trip(restore_tuning):
    t = P.set_tuning(small_max_deg=8, small_ctas_per_sm=3, warp_ctas_per_sm=32,
                     admit_ctas_per_sm=1, concurrent=0, pdl=0, fused_admission=1,
                     contract_table_slots=4096, ip_trial_group=3, contract_merge=1)
    assert t.to_dict() == dict(small_max_deg=8, small_ctas_per_sm=3, warp_ctas_per_sm=32,
                               admit_ctas_per_sm=1, concurrent=0, pdl=0, fused_admission=1,
                               contract_table_slots=4096, ip_trial_group=3, contract_merge=1)


# ------------------------------------------------------------------ GPU
def _batch():
    """R-MAT rows of every length (1..8, 9..16, 17..128, longer), a geometric
    graph, a weighted graph and a star (one hub of degree 2999)."""
    gs = [(gg.rmat(11 + i % 3, 8, 70 + i), [2, 5, 16][i % 3]) for i in range(4)]
    gs += [(gg.rgg2d(4000, 71), 8),
           (gg.random_weights(gg.rmat(11, 8, 72), 73, max_node_w=4, max_edge_w=7), 4),
           (gg.star(3000), 2)]
    return gs


SETTINGS = [
    dict(small_max_deg=8),
    dict(small_ctas_per_sm=1, warp_ctas_per_sm=1, admit_ctas_per_sm=1),
    dict(small_ctas_per_sm=32, warp_ctas_per_sm=32, admit_ctas_per_sm=64),
    dict(concurrent=0),
    dict(pdl=0),
    dict(concurrent=0, pdl=0),
    dict(small_max_deg=8, small_ctas_per_sm=2, warp_ctas_per_sm=3, admit_ctas_per_sm=5,
         concurrent=0),
    dict(fused_admission=1),
    dict(fused_admission=1, admit_ctas_per_sm=1, concurrent=0),
    dict(contract_merge=1),               # contraction by member lists and merges
    dict(contract_merge=1, contract_table_slots=4096),   # merges where they fit, else passes
    dict(contract_table_slots=4096),      # contraction in passes of 4096 slots
    dict(contract_table_slots=1),         # a pass per coarse node
    dict(ip_trial_group=1),               # initial-partitioning trials one at a time
    dict(ip_trial_group=5),               # groups of 5, 5, 5 and 1 of the 16 trials
]


@pytest.mark.gpu
@pytest.mark.parametrize("si", range(len(SETTINGS)))
def test_results_do_not_depend_on_the_tuning(restore_tuning, si):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    gs = _batch()
    P.set_tuning(**{**DEFAULT, **SETTINGS[si]})
    items = [dict(row_ptr=torch.from_numpy(g.row_ptr).to(dev), col=torch.from_numpy(g.col).to(dev),
                  node_w=torch.from_numpy(g.node_w).to(dev), edge_w=torch.from_numpy(g.edge_w).to(dev),
                  k=k, eps=0.03, seed=11 + i) for i, (g, k) in enumerate(gs)]
    for graph_rounds in (0, 1):
        res = P.sclap_partition_batch(items, device=True,
                                      cfg=P.default_config(graph_rounds=graph_rounds))
        for i, (g, k) in enumerate(gs):
            ref = O.partition(g, k, 0.03, seed=11 + i)
            assert (res[i].status, res[i].cut) == (ref.status, ref.cut), (i, graph_rounds)
            assert np.array_equal(res[i].block.cpu().numpy(), ref.block), (i, graph_rounds)


@pytest.mark.gpu
def test_autotune_installs_a_valid_setting_with_unchanged_results(restore_tuning):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    gs = _batch()
    P.set_tuning(**DEFAULT)
    items = [dict(row_ptr=torch.from_numpy(g.row_ptr).to(dev), col=torch.from_numpy(g.col).to(dev),
                  k=k, eps=0.03, seed=5 + i) for i, (g, k) in enumerate(gs)]
    before = P.sclap_partition_batch(items, device=True)
    t = P.autotune(items, reps=1)
    assert P.get_tuning().to_dict() == t.to_dict()
    assert t.small_max_deg in (8, 16) and t.concurrent in (0, 1)
    after = P.sclap_partition_batch(items, device=True)
    for x, y in zip(before, after):
        assert (x.status, x.cut) == (y.status, y.cut)
        assert np.array_equal(x.block.cpu().numpy(), y.block.cpu().numpy())


def _bucket_mix_graph():
    """A path of 110,000 nodes (degree 2: the degree <= 4 bucket needs 430
    blocks of 256 nodes), one node of degree 6 and one of degree 12 (one
    node each in the degree 5..8 and 9..16 buckets)."""
    n_path = 110_000
    s = [np.arange(n_path - 1)]
    d = [np.arange(1, n_path)]
    c6, c12 = n_path, n_path + 7
    s += [np.full(6, c6), np.full(12, c12)]
    d += [np.arange(c6 + 1, c6 + 7), np.arange(c12 + 1, c12 + 13)]
    return gg.from_edges(c12 + 13, np.concatenate(s), np.concatenate(d), name="bucket-mix")


@pytest.mark.gpu
def test_thread_launch_split_serves_every_small_bucket(restore_tuning):
    """With one CTA per SM the thread-per-node launch has fewer blocks than
    the three small buckets need; the split must still give the two
    single-node buckets a block each (rounding both up to one once took the
    last bucket's block away, so its node never proposed)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    g = _bucket_mix_graph()
    deg = g.degrees()
    assert (deg <= 4).sum() > 2 * 152 * 256 and ((deg > 4) & (deg <= 8)).sum() == 1
    assert ((deg > 8) & (deg <= 16)).sum() == 1
    P.set_tuning(**{**DEFAULT, "small_ctas_per_sm": 1})
    label = np.arange(g.n, dtype=np.int32)
    W = np.ones(g.n, np.int64)
    for U, rkey in ((3, 5), (20, 99)):
        ol, oW, om, on = O.lp_round(g, O.MODE_CLUSTER, label, W, U, rkey, 1, want_next=True)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        tl, tW = t(label), t(W)
        an = torch.zeros(g.n, dtype=torch.uint8, device=dev)
        moved = P.sclap_lp_round(0, t(g.row_ptr), t(g.col), t(g.node_w), t(g.edge_w), tl, tW, U,
                                 rkey, 1, active_next=an)
        assert moved == om
        assert np.array_equal(tl.cpu().numpy(), ol)
        assert np.array_equal(tW.cpu().numpy(), oW)
        assert np.array_equal(an.cpu().numpy(), on)
        # both centres move in the oracle (each joins a singleton leaf), so a
        # centre left without a proposal would show as a difference above
        assert ol[110_000] != 110_000 and ol[110_007] != 110_007


def _canon(rp, col, w):
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    o = np.lexsort((col, src))
    return src[o], col[o], w[o]


@pytest.mark.gpu
@pytest.mark.parametrize("slots", [1, 64, 4096])
def test_contraction_in_passes_equals_the_oracle(restore_tuning, slots):
    """A contraction table capped at `slots` slots per pass (1: a pass per
    coarse node) builds the same coarse graph as the oracle: map, node
    weights, row offsets, and the arcs of every row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    g = gg.random_weights(gg.rmat(13, 8, 3), 5)
    P.set_tuning(**{**DEFAULT, "contract_table_slots": slots})
    for label in (O.cluster(g, 40, seed=2)[0],
                  np.random.default_rng(4).integers(0, g.n // 30, g.n).astype(np.int32)):
        c = O.contract(g, label)
        cmap, crp, ccol, cnw, cew = P.sclap_contract(t(g.row_ptr), t(g.col), t(g.node_w),
                                                     t(g.edge_w), t(label))
        assert np.array_equal(cmap.cpu().numpy(), c.cmap)
        assert np.array_equal(cnw.cpu().numpy(), c.node_w)
        assert np.array_equal(crp.cpu().numpy(), c.row_ptr)
        a = _canon(crp.cpu().numpy(), ccol.cpu().numpy(), cew.cpu().numpy())
        b = _canon(c.row_ptr, c.col, c.edge_w)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def _grid_blocks(rows, cols, bh, bw):
    r, c = np.divmod(np.arange(rows * cols), cols)
    return ((r // bh) * -(-cols // bw) + c // bw).astype(np.int32)


@pytest.mark.gpu
@pytest.mark.parametrize("merge", [1, 0])
def test_contraction_by_merges_covers_every_class(restore_tuning, merge):
    """Grid blocks give coarse nodes of each merge class: 10x10 blocks (40
    inter-cluster arcs, 400 member arcs: a warp each), 40x40 (160 and 6,400:
    a CTA each), 50-row strips (400 inter-cluster arcs but 40,000 member
    arcs: large), and a star whose centre is a cluster of its own (4,999
    inter-cluster arcs: large).  Same coarse graph as the oracle with merges
    on or off."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    P.set_tuning(**{**DEFAULT, "contract_merge": merge})
    grid = gg.random_weights(gg.grid(200, 200), 8)
    star = gg.random_weights(gg.star(4999), 9)
    cases = [(grid, _grid_blocks(200, 200, 10, 10)), (grid, _grid_blocks(200, 200, 40, 40)),
             (grid, _grid_blocks(200, 200, 50, 200)),
             (grid, np.where(np.arange(40000) < 36000, 0, np.arange(40000)).astype(np.int32)),
             (star, np.where(np.arange(5000) == 0, 0, 1 + np.arange(5000) % 7).astype(np.int32))]
    for g, label in cases:
        c = O.contract(g, label)
        cmap, crp, ccol, cnw, cew = P.sclap_contract(t(g.row_ptr), t(g.col), t(g.node_w),
                                                     t(g.edge_w), t(label))
        assert np.array_equal(cmap.cpu().numpy(), c.cmap)
        assert np.array_equal(cnw.cpu().numpy(), c.node_w)
        assert np.array_equal(crp.cpu().numpy(), c.row_ptr)
        a = _canon(crp.cpu().numpy(), ccol.cpu().numpy(), cew.cpu().numpy())
        b = _canon(c.row_ptr, c.col, c.edge_w)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)

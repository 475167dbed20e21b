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
               concurrent=1, pdl=1)


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
                                       ("concurrent", -1), ("pdl", 2)])
def test_out_of_range_values_are_rejected_and_leave_the_setting(restore_tuning, field, bad):
    P.set_tuning(**DEFAULT)
    with pytest.raises(P.SclapError) as e:
        P.set_tuning(**{field: bad})
    assert e.value.code == P.EINVAL
    assert P.get_tuning().to_dict() == DEFAULT


def test_set_tuning_round_trip(restore_tuning):
    t = P.set_tuning(small_max_deg=8, small_ctas_per_sm=3, warp_ctas_per_sm=32,
                     admit_ctas_per_sm=1, concurrent=0, pdl=0)
    assert t.to_dict() == dict(small_max_deg=8, small_ctas_per_sm=3, warp_ctas_per_sm=32,
                               admit_ctas_per_sm=1, concurrent=0, pdl=0)


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

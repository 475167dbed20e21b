"""sclap_cut_static, the entry point that works without device allocation,
against sclap_cut on the same inputs.

Collected last on purpose: it must give the same answers in a fresh process
and after every other GPU test has run (and left the allocator pools and
the library's state behind it).
"""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1402_3281_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


def dt(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).to(DEV)


def _graphs():
    return [
        gg.random_weights(gg.rmat(12, 8, 5), 3, max_node_w=6, max_edge_w=9),
        gg.rgg2d(3000, 4),
        gg.star(5000),
    ]


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("k", [1, 2, 37, P.CUT_STATIC_MAX_K])
def test_two_calls_in_a_row_match_sclap_cut(gi, k):
    g = _graphs()[gi]
    if k > g.n:
        pytest.skip("k above n")
    rp, col, nw, ew = dt(g.row_ptr), dt(g.col), dt(g.node_w), dt(g.edge_w)
    rng = np.random.default_rng(1000 * gi + k)
    # two different partitions back to back: the second call must not see
    # anything left in the scratch by the first
    for _ in range(2):
        blk = rng.integers(0, k, g.n).astype(np.int32)
        b = dt(blk)
        cut_s, bw = P.sclap_cut_static(rp, col, nw, ew, b, k)
        cut_ref = P.sclap_cut(rp, col, ew, b)
        assert cut_s == cut_ref
        expect = np.bincount(blk, weights=g.node_w.astype(np.int64), minlength=k).astype(np.int64)
        assert np.array_equal(bw, expect)
    torch.cuda.synchronize()


def test_unit_weights_and_repeat_identical():
    g = gg.rmat(11, 8, 2)
    rp, col = dt(g.row_ptr), dt(g.col)
    blk = dt(np.random.default_rng(3).integers(0, 16, g.n).astype(np.int32))
    first = P.sclap_cut_static(rp, col, None, None, blk, 16)
    second = P.sclap_cut_static(rp, col, None, None, blk, 16)
    assert first[0] == second[0] == P.sclap_cut(rp, col, None, blk)
    assert np.array_equal(first[1], second[1])
    assert int(first[1].sum()) == g.n


def test_rejects_k_above_the_limit_and_labels_out_of_range():
    g = gg.rmat(13, 8, 1)
    rp, col = dt(g.row_ptr), dt(g.col)
    blk = dt(np.zeros(g.n, np.int32))
    with pytest.raises(P.SclapError) as e:
        P.sclap_cut_static(rp, col, None, None, blk, P.CUT_STATIC_MAX_K + 1)
    assert e.value.code == P.EINVAL
    bad = np.zeros(g.n, np.int32)
    bad[g.n // 2] = 5
    with pytest.raises(P.SclapError) as e:
        P.sclap_cut_static(rp, col, None, None, dt(bad), 5)
    assert e.value.code == P.EINVAL
    # the scratch is usable again right after a rejected call
    cut, bw = P.sclap_cut_static(rp, col, None, None, blk, 1)
    assert cut == 0 and int(bw[0]) == g.n

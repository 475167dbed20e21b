"""sclap_cut_static, the entry point that works without device allocation,
checked against an independent recount (the CPU oracle's cut and NumPy
block weights) and against sclap_cut on the same inputs.

Collected last on purpose: in the usual run it executes after every other
GPU test, in the same process, with the allocator pools and the library's
state those tests leave behind; it also passes when run alone in a fresh
process (pytest tests/test_zz_no_alloc.py).
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


def _graphs():
    # every graph has at least SCLAP_CUT_STATIC_MAX_K = 4096 nodes, so the
    # largest k runs on each of them
    return [
        gg.random_weights(gg.rmat(12, 8, 5), 3, max_node_w=6, max_edge_w=9),
        gg.rgg2d(5000, 4),
        gg.star(5000),
    ]


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("k", [1, 2, 37, P.CUT_STATIC_MAX_K])
def test_two_calls_in_a_row_match_a_recount_and_sclap_cut(gi, k):
    g = _graphs()[gi]
    assert k <= g.n
    rp, col, nw, ew = dt(g.row_ptr), dt(g.col), dt(g.node_w), dt(g.edge_w)
    rng = np.random.default_rng(1000 * gi + k)
    # two different partitions back to back: the second call must not see
    # anything left in the scratch by the first
    for _ in range(2):
        blk = rng.integers(0, k, g.n).astype(np.int32)
        b = dt(blk)
        cut_s, bw = P.sclap_cut_static(rp, col, nw, ew, b, k)
        assert cut_s == O.cut(g, blk)                      # CPU oracle's cut
        assert cut_s == P.sclap_cut(rp, col, ew, b)        # the allocating entry point
        expect = np.bincount(blk, weights=g.node_w.astype(np.int64), minlength=k).astype(np.int64)
        assert np.array_equal(bw, expect)
    torch.cuda.synchronize()


def test_unit_weights_and_repeat_identical():
    g = gg.rmat(11, 8, 2)
    rp, col = dt(g.row_ptr), dt(g.col)
    host = np.random.default_rng(3).integers(0, 16, g.n).astype(np.int32)
    blk = dt(host)
    first = P.sclap_cut_static(rp, col, None, None, blk, 16)
    second = P.sclap_cut_static(rp, col, None, None, blk, 16)
    assert first[0] == second[0] == O.cut(g, host)
    assert np.array_equal(first[1], second[1])
    assert np.array_equal(first[1], np.bincount(host, minlength=16))


def test_calls_take_no_device_memory():
    """The promise of the entry point: after the first call (which looks up
    the scratch array's address), further calls change the device's free
    memory by nothing."""
    g = gg.rgg2d(20000, 9)
    rp, col, nw, ew = dt(g.row_ptr), dt(g.col), dt(g.node_w), dt(g.edge_w)
    blks = [dt(np.random.default_rng(s).integers(0, 64, g.n).astype(np.int32)) for s in range(4)]
    P.sclap_cut_static(rp, col, nw, ew, blks[0], 64)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for b in blks:
        P.sclap_cut_static(rp, col, nw, ew, b, 64)
        P.sclap_cut_static(rp, col, None, None, b, 64)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


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

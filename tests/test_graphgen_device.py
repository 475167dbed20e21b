"""The device-side R-MAT generator (graphgen.device), run with CPU tensors:
exact SplitMix64, a valid canonical CSR, results independent of chunk and
part sizes, a bijective id permutation, and the same model as the NumPy
generator (edge counts and degree skew close)."""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")

from graphgen.device import _permute, _s64, _splitmix64_t, rmat_torch, splitmix64_py  # noqa: E402


def test_splitmix64_tensor_equals_exact_reference():
    # published test value: the first output of a SplitMix64 stream seeded
    # with 0 (state 0x9E3779B97F4A7C15 through the output function)
    assert splitmix64_py(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    rng = np.random.default_rng(1)
    xs = [int(x) for x in rng.integers(0, 2**63, 4000, dtype=np.uint64)]
    xs += [0, 1, 2**63, 2**64 - 1, 0x9E3779B97F4A7C15]
    out = _splitmix64_t(torch.tensor([_s64(x) for x in xs], dtype=torch.int64)).tolist()
    assert [o & (2**64 - 1) for o in out] == [splitmix64_py(x) for x in xs]


@pytest.mark.parametrize("scale", [1, 2, 5, 9, 14])
def test_permutation_is_a_bijection(scale):
    x = torch.arange(1 << scale, dtype=torch.int64)
    y = _permute(x, scale, 12345)
    assert torch.equal(torch.sort(y).values, x)


@pytest.mark.parametrize("scale,ef,seed", [(6, 4, 0), (9, 8, 1), (11, 16, 2)])
def test_valid_canonical_csr(scale, ef, seed):
    rp, col = rmat_torch(scale, ef, seed)
    assert rp.dtype == torch.int64 and col.dtype == torch.int32
    n = rp.numel() - 1
    g = gg.Graph(rp.numpy(), col.numpy(), np.ones(n, np.int32), np.ones(col.numel(), np.int32))
    gg.validate(g)      # symmetric, no self-loops, no duplicates, sorted rows


def test_chunk_and_part_sizes_do_not_change_the_graph():
    ref = rmat_torch(10, 8, 7)
    for chunk, parts in [(1 << 10, 1), (777, 3), (1 << 20, 16)]:
        rp, col = rmat_torch(10, 8, 7, edge_chunk=chunk, parts=parts)
        assert torch.equal(rp, ref[0]) and torch.equal(col, ref[1])


def test_seeds_differ_and_repeat():
    a = rmat_torch(9, 8, 0)
    b = rmat_torch(9, 8, 0)
    c = rmat_torch(9, 8, 1)
    assert torch.equal(a[1], b[1])
    assert not (a[0].numel() == c[0].numel() and torch.equal(a[1], c[1]))


def test_same_model_as_the_numpy_generator():
    rp, col = rmat_torch(13, 8, 0)
    deg = (rp[1:] - rp[:-1]).numpy()
    h = gg.rmat(13, 8, 0)
    assert abs(col.numel() - h.arcs) < 0.02 * h.arcs
    # heavy-tailed like the reference: similar maximum degree and share of
    # degree-0 nodes
    assert 0.7 < deg.max() / h.degrees().max() < 1.4
    assert abs((deg == 0).mean() - (h.degrees() == 0).mean()) < 0.02

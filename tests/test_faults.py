"""Failure paths of the library, injected on the host (sclap_debug_inject):
a bounded device-side wait that runs out, a hash-table probe limit that is
reached, a device allocation that fails.  Each is reported as its error
code and the library is usable, and bit-exact with the oracle, on the next
call.  Nothing here faults, traps or hangs the GPU: the waits are bounded
and only their bound is lowered.

The CPU test checks the argument validation of the injection call itself
(it makes no device call)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import paper_1402_3281_gb300 as P


def test_injection_arguments_are_validated():
    for bad in (dict(wait_limit=-1), dict(probe_limit=-1), dict(fail_allocs=-1),
                dict(wait_limit=1 << 32), dict(probe_limit=1 << 33)):
        with pytest.raises(P.SclapError) as e:
            P.debug_inject(**bad)
        assert e.value.code == P.EINVAL
    P.debug_inject()          # all zeros: defaults


# ------------------------------------------------------------------ GPU
@pytest.fixture
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    yield torch.device("cuda:0")
    P.debug_inject()          # defaults again, whatever the test did


def _dg(g, dev):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t(g.row_ptr), t(g.col), t(g.node_w), t(g.edge_w)


def _check_equals_oracle(g, k, seed, dev, cfg=None):
    ref = O.partition(g, k, 0.03, seed=seed)
    res = P.sclap_partition_device(*_dg(g, dev), k=k, eps=0.03, seed=seed, cfg=cfg)
    assert (res.status, res.cut) == (ref.status, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block)


@pytest.fixture
def fused():
    before = P.get_tuning().to_dict()
    P.set_tuning(fused_admission=1)
    yield
    P.set_tuning(**before)


@pytest.mark.gpu
@pytest.mark.parametrize("graph_rounds", [0, 1])
def test_wait_that_runs_out_reports_timeout(dev, fused, graph_rounds):
    """With the admission as one cooperative launch, its grid barriers allow
    one poll: CTAs that arrive before the last one give up, set the timeout
    bit and leave; later launches of the run see the bit and do nothing.
    The call returns SCLAP_ETIMEOUT; the next call with the default limit is
    bit-exact."""
    g = gg.rmat(16, 8, 0)
    cfg = P.default_config(graph_rounds=graph_rounds)
    P.debug_inject(wait_limit=1)
    with pytest.raises(P.SclapError) as e:
        P.sclap_partition_device(*_dg(g, dev), k=8, eps=0.03, seed=0, cfg=cfg)
    assert e.value.code == P.ETIMEOUT
    P.debug_inject()
    _check_equals_oracle(g, 8, 0, dev, cfg=cfg)


@pytest.mark.gpu
def test_probe_limit_reports_internal_error(dev):
    """One probe per insertion: the first collision in a warp or CTA table
    of the clustering sweep leaves an arc unplaced, which is reported as
    SCLAP_EINTERNAL instead of a silently wrong partition."""
    g = gg.rmat(14, 8, 1)
    P.debug_inject(probe_limit=1)
    with pytest.raises(P.SclapError) as e:
        P.sclap_partition_device(*_dg(g, dev), k=4, eps=0.03, seed=2)
    assert e.value.code == P.EINTERNAL
    P.debug_inject()
    _check_equals_oracle(g, 4, 2, dev)


@pytest.mark.gpu
def test_failed_device_allocation_reports_enomem(dev):
    g = gg.rgg2d(3000, 5)
    for nth in (1, 3, 40):          # the first, an early and a later allocation fail
        P.debug_inject(fail_allocs=nth)
        with pytest.raises(P.SclapError) as e:
            P.sclap_partition(g.row_ptr, g.col, k=4, eps=0.03, seed=1)
        assert e.value.code == P.ENOMEM
        P.debug_inject()
    res = P.sclap_partition(g.row_ptr, g.col, k=4, eps=0.03, seed=1)
    ref = O.partition(g, 4, 0.03, seed=1)
    assert res.cut == ref.cut and np.array_equal(res.block, ref.block)


@pytest.mark.gpu
def test_failed_allocation_in_the_server_comes_back_through_poll(dev):
    g = gg.rmat(11, 8, 4)
    with P.Server(workers=1) as srv:
        P.debug_inject(fail_allocs=1)
        rid = srv.submit(g.row_ptr, g.col, k=4)
        with pytest.raises(P.SclapError) as e:
            srv.poll(rid, -1)
        assert e.value.code == P.ENOMEM
        P.debug_inject()
        ok = srv.submit(g.row_ptr, g.col, k=4)      # the server keeps serving
        res = srv.poll(ok, -1)
        ref = O.partition(g, 4, 0.03, seed=0)
        assert res.status == P.OK and res.cut == ref.cut
        assert np.array_equal(res.block, ref.block)

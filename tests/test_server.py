"""The serving loop (sclap_server_*): requests submitted from several host
threads while batches are on the GPU come back bit-identical to the same
requests partitioned alone, under any admission budget; request errors come
back through poll."""
import random
import threading
import time

import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1402_3281_gb300 as P  # noqa: E402


def _requests(count, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i % 3 == 0:
            g = gg.rmat(int(rng.integers(8, 13)), 8, seed * 100 + i)
        elif i % 3 == 1:
            g = gg.rgg2d(int(rng.integers(300, 6000)), seed * 100 + i)
        else:
            g = gg.random_weights(gg.rmat(int(rng.integers(8, 11)), 8, i), i, 4, 6)
        k = int(rng.choice([2, 3, 8, 16, 64]))
        k = min(k, g.n)
        eps = float(rng.choice([0.01, 0.03, 0.05]))
        out.append((g, k, eps, int(rng.integers(0, 2**40))))
    return out


def _alone(req):
    g, k, eps, seed = req
    return P.sclap_partition(g.row_ptr, g.col, g.node_w, g.edge_w, k=k, eps=eps, seed=seed)


def _serve(reqs, threads=3, **opts):
    """Submit from several threads with random gaps; poll in order."""
    ids = [None] * len(reqs)
    with P.Server(**opts) as srv:
        def feeder(part):
            r = random.Random(part[0] if part else 0)
            for i in part:
                g, k, eps, seed = reqs[i]
                ids[i] = srv.submit(g.row_ptr, g.col, g.node_w, g.edge_w, k, eps, seed)
                time.sleep(r.random() * 0.004)
        parts = [list(range(t, len(reqs), threads)) for t in range(threads)]
        ts = [threading.Thread(target=feeder, args=(p,)) for p in parts]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        return [srv.poll(rid, -1) for rid in ids]


@pytest.mark.parametrize("opts", [
    dict(),                                              # defaults: 2 workers
    dict(workers=4, max_batch=5),                        # many small batches in flight
    dict(workers=2, device_budget_bytes=1 << 24),        # tight budget: near one at a time
    dict(workers=1, max_batch=64, linger_us=3000),       # one worker, lingering batches
])
def test_served_results_equal_alone(opts):
    reqs = _requests(24, seed=len(opts))
    got = _serve(reqs, **opts)
    for req, res in zip(reqs, got):
        ref = _alone(req)
        assert res.status == ref.status
        assert res.cut == ref.cut
        assert np.array_equal(res.block, ref.block)
        assert res.max_block_weight == ref.max_block_weight
        assert res.latency_ms > 0


def test_poll_pending_unknown_and_errors():
    g = gg.rmat(11, 8, 3)
    with P.Server(workers=1) as srv:
        rid = srv.submit(g.row_ptr, g.col, k=4)
        res = srv.poll(rid, 0)
        while res is None:
            res = srv.poll(rid, 5)
        assert res.status == P.OK
        with pytest.raises(P.SclapError) as e:       # released after a completed poll
            srv.poll(rid, 0)
        assert e.value.code == P.EINVAL
        with pytest.raises(P.SclapError) as e:       # k > n: rejected at submit
            srv.submit(g.row_ptr, g.col, k=g.n + 1)
        assert e.value.code == P.EINVAL
        bad = g.col.copy()
        bad[5] = g.n + 7                             # neighbour out of range
        rid = srv.submit(g.row_ptr, bad, k=2)
        with pytest.raises(P.SclapError) as e:       # found by validation on the device
            srv.poll(rid, -1)
        assert e.value.code == P.ECSR
        ok = srv.submit(g.row_ptr, g.col, k=2)        # the server keeps serving
        assert srv.poll(ok, -1).status == P.OK


def test_budget_smaller_than_a_request_is_rejected():
    g = gg.rmat(12, 8, 1)
    with P.Server(device_budget_bytes=1 << 16) as srv:
        with pytest.raises(P.SclapError) as e:
            srv.submit(g.row_ptr, g.col, k=2)
        assert e.value.code == P.ENOMEM


def test_destroy_with_queued_requests():
    reqs = _requests(12, seed=9)
    srv = P.Server(workers=1, max_batch=2)
    for g, k, eps, seed in reqs:
        srv.submit(g.row_ptr, g.col, g.node_w, g.edge_w, k, eps, seed)
    srv.close()   # stops after the running batch; queued requests are dropped

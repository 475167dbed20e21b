"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank gets its own batch seed and the timed value is the maximum over ranks.
The partitioner itself has no cross-rank exchange (replicas only)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wsz, r, lr = bench.dist_env()
        mx = bench.max_over_ranks(10.0 + 5 * rank, wsz)
        dist.barrier()
        out[rank] = (r, lr, wsz, mx, bench.rank_seed(r))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_and_distinct_seeds():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(ws):
        rank, local, wsz, mx, seed = res[r]
        assert (rank, local, wsz) == (r, r, ws)
        assert mx == 15.0
    assert res[0][4] != res[1][4]


def test_single_rank_is_plain():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5

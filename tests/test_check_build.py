"""The bounds-check build (compiled with -DSCLAP_CHECK=1: libsclap_check.so).

In that build every data-dependent index the kernels use (a neighbour, a
label, a coarse id, a hub's direct entry) is checked against its array's
length first; an index out of range is never used and the call fails with
SCLAP_EINTERNAL.  The GPU test builds it, then in a child process (the
library is chosen when the binding loads, through SCLAP_LIBRARY) runs the
check's self test and partitions graphs that reach every kernel family —
thread, warp, CTA and hub propose, heavy-row contraction, grouped growing,
the marking queue of moved long rows, a batch of several graphs — each
checked against the oracle: no check may fire and every result must equal
the normal build's.
"""
import os
import subprocess
import sys

import pytest

import paper_1402_3281_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import graphgen as gg
import oracle as O
import paper_1402_3281_gb300 as P
from test_gpu_parity import hub_graph, split_hub_graph

assert P.check_build(), "not the bounds-check build"
P.check_selftest()
dev = torch.device("cuda:0")
t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
cases = [(gg.rmat(12, 8, 3), 4), (gg.random_weights(gg.rmat(11, 8, 4), 7), 5),
         (hub_graph(2), 8), (split_hub_graph(3), 16), (gg.rgg2d(5000, 2), 2)]
for g, k in cases:
    res = P.sclap_partition_device(t(g.row_ptr), t(g.col), t(g.node_w), t(g.edge_w), k=k,
                                   eps=0.03, seed=1)
    ref = O.partition(g, k, 0.03, seed=1)
    assert (res.status, res.cut) == (ref.status, ref.cut), (g.name, k, res.cut, ref.cut)
    assert np.array_equal(res.block.cpu().numpy(), ref.block), (g.name, k)
items = [dict(row_ptr=t(g.row_ptr), col=t(g.col), node_w=t(g.node_w), edge_w=t(g.edge_w),
              k=k, eps=0.03, seed=7 + i) for i, (g, k) in enumerate(cases)]
out = P.sclap_partition_batch(items, device=True)
for i, (g, k) in enumerate(cases):
    ref = O.partition(g, k, 0.03, seed=7 + i)
    assert (out[i].status, out[i].cut) == (ref.status, ref.cut), (g.name, k)
g = split_hub_graph(3)
label, _ = O.cluster(g, 40, seed=2)
c = O.contract(g, label)
cmap, crp, ccol, cnw, cew = P.sclap_contract(t(g.row_ptr), t(g.col), t(g.node_w), t(g.edge_w),
                                             t(label))
assert np.array_equal(cmap.cpu().numpy(), c.cmap)
assert np.array_equal(crp.cpu().numpy(), c.row_ptr)
torch.cuda.synchronize()
print("CHECK-OK")
"""


def test_normal_build_is_not_a_check_build():
    assert not P.check_build()
    with pytest.raises(P.SclapError) as e:
        P.check_selftest()
    assert e.value.code == P.EINVAL


@pytest.mark.gpu
def test_bounds_check_build_runs_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1402_3281_gb300 import build as B
    so = B.build(check=True)
    env = dict(os.environ, SCLAP_LIBRARY=so)
    script = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True,
                       timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "CHECK-OK" in r.stdout

"""The benchmark's reference arm (the CPU oracle) keeps the JSON contract
(no GPU needed): one line with the metric, the oracle as cpu_baseline, an
end-to-end figure without copies; ranks other than 0 print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--count", "16"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "partitions/s" and d["unit"] == "partitions/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert isinstance(d["config"]["workload"], str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_other_ranks_print_nothing():
    assert _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}) == []


def test_propose_roofline_arithmetic():
    """The sweep's roofline from a library profile: 12 B per weighted arc, 8
    per unit-weight arc, 44 per listed node, over the phases' time; the
    sector reading adds 28 B per arc (a 4-byte label gather read as a 32-byte
    sector); traffic scales the committed bytes per arc to the average
    phase when the capture matches the current kernel source."""
    sys.path.insert(0, ROOT)
    import bench
    prof = {"propose_arcs": [600, 300, 100, 0], "propose_arcs_unit": 400,
            "propose_nodes": [50, 30, 20, 0], "sweep_ms": 2.0, "sweeps": 4,
            "propose_ms": [1.0, 0.5, 0.5, 0.0], "propose_launches": [4, 4, 4, 0]}
    r = bench.propose_roofline(prof, prof_ms=8.0, steps=2)
    alg = 12 * 600 + 8 * 400 + 44 * 100
    assert abs(r["achieved"] - alg / 2e-3 / 1e9) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert abs(r["sector_model"]["achieved"] - (alg + 28 * 1000) / 2e-3 / 1e9) < 1e-12
    assert r["launches"] == 4 and abs(r["avg_launch_ms"] - 0.5) < 1e-15
    assert abs(r["bytes_per_launch"] - alg / 4) < 1e-9
    assert abs(r["share_of_step"] - 0.25) < 1e-15 and abs(r["profiled_ms_per_step"] - 4.0) < 1e-15
    tr = bench.traffic_for(os.path.join(ROOT, "paper_1402_3281_gb300", "csrc", "lp.cu"))
    if tr is not None and tr[0]:
        assert abs(r["traffic"] - tr[0] * 1000 / 4) < 1e-6
    else:
        assert r["traffic"] is None


def test_sweep_by_kind_groups_the_sub_round_records():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    # (kind, round, class, nodes, arcs, propose ms, admission ms)
    ph = np.array([[0, 0, 0, 10, 100, 1.0, 0.5], [0, 0, 1, 20, 300, 1.0, 0.5],
                   [1, 0, 0, 5, 50, 0.5, 0.1]], dtype=np.float64)
    out = bench.sweep_by_kind(ph, steps=1)
    assert set(out) == {bench.KINDS.get(0, "0"), bench.KINDS.get(1, "1")}
    c = out[bench.KINDS.get(0, "0")]
    assert c["sub_rounds"] == 2 and c["nodes"] == 30 and c["arcs"] == 400 and c["sweep_ms"] == 2.0
    assert abs(c["edges_per_s"] - 400 / 2e-3) < 1e-6
    assert abs(c["gbs"] - (12 * 400 + 44 * 30) / 2e-3 / 1e9) < 1e-12
    assert bench.sweep_by_kind(np.zeros((0, 7))) == {}

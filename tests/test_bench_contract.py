"""The benchmark's reference arm (the CPU oracle timed on a bounded sample) runs without a GPU
and prints one JSON line with the keys the benchmark contract fixes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "active-edge updates/s" and d["unit"] == "updates/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("cube3d_128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_dram_rate():
    sys.path.insert(0, ROOT)
    import bench
    # 39.1 GB in 34.1 ms and 42.9 GB in 46.5 ms: 1146.6 and 922.6 GB/s, mean 1034.6
    r = bench.dram_rate([39.1e9, 42.9e9], [34.1, 46.5])
    assert abs(r - (39.1 / 0.0341 + 42.9 / 0.0465) / 2) < 1e-6
    import pytest
    with pytest.raises(ValueError):
        bench.dram_rate([1.0], [1.0, 2.0])


def test_cpu_baseline_batched_on_tiny_instances():
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1511_06441_gb300 import synth
    insts = [synth.random_small_instance(s, max_vertices=30) for s in range(12)]
    ups = [oracle.cycle(i.extents, i.f1, i.f2, i.A, i.B, i.M, trace=False).updates for i in insts]
    out = bench.cpu_baseline_batched(insts, ups, budget_updates=sum(ups), cap_updates=max(ups), cores=2)
    assert out["kind"] == "oracle" and out["cores"] == 2 and out["value"] > 0
    assert out["whole_batch_instances_per_s_estimate"] > 0 and "12 of 12" in out["sample"]

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


def test_algorithmic_bytes_and_roofline_block():
    sys.path.insert(0, ROOT)
    import bench
    # 8 B per update, 13 per arrival, 6 per edge slot of an improved vertex, 12 per started flow
    assert bench.alg_bytes(6, 10, 2, 3, 4) == 80 + 26 + 108 + 48
    rec = [0] * 16
    rec[7], rec[13], rec[14], rec[8] = 10, 2, 3, 4
    assert bench.alg_bytes_of(6, rec) == 262
    r = bench.roofline_block(2e9, 0.5, "k", traffic=3e9)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 4.0) < 1e-12 and r["frac"] == r["achieved"] / r["peak"]
    assert abs(r["dram_gbs"] - 6.0) < 1e-12 and r["unit"] == "GB/s"


def test_summary_repeats_the_section_headlines():
    sys.path.insert(0, ROOT)
    import bench
    line = {"value": 5.0, "roofline": {"frac": 0.1}, "e2e": {"value": 4.0},
            "engines": {"event_vs_sweep": 0.3},
            "batched": {"instances_per_s": 30.0, "plain_instances_per_s": 15.0, "speedup_vs_plain": 2.0,
                        "agree_with_plain": 512, "roofline": {"frac": 0.2}},
            "serving": {"queries": 10, "rates": [
                {"rate_x_saturation": 0.5, "served": {"p99_ms": 3.0, "equal_to_alone": 10}, "plain": {"p99_ms": 4.0}},
                {"rate_x_saturation": 1.0, "served": {"p99_ms": 5.0, "equal_to_alone": 9}, "plain": {"p99_ms": 4.0}}]}}
    s = bench.summary(line)
    assert s["updates_per_s"] == 5.0 and s["batched"]["speedup_vs_plain"] == 2.0
    assert s["serving"]["served_p99_le_plain_everywhere"] is False and s["serving"]["equal_to_alone"] == 9
    assert s["event_form_vs_sweep"] == 0.3


def test_traffic_record_from_an_ncu_csv(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
           '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = []
    for i, (rd, wr, t) in enumerate([(1, 2, 10), (10, 20, 100), (3, 4, 30), (30, 40, 300), (5, 6, 50), (50, 60, 500)]):
        for m, v in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr), ("gpu__time_duration.sum", t)):
            rows.append(f'"{i}","1","python","h","k_event","1","7","(512, 1, 1)","(304, 1, 1)","0","10.3",'
                        f'"Command line profiler metrics","{m}","byte","{v:,}"\n')
    csv = tmp_path / "t.csv"
    csv.write_text("==PROF== noise\n" + head + "".join(rows))
    rec = bench.record_traffic(str(csv), "k_event_cube128_traffic.json", "cmd", out_dir=str(tmp_path))
    assert rec["traffic_bytes_per_launch"] == {"400": 30.0, "800": 70.0, "1600": 110.0}  # launches 1, 3, 5
    assert rec["duration_ns_under_ncu"]["1600"] == 500.0
    assert rec["kernel_source_sha256"] == bench._kernel_sha(bench.TRAFFIC["k_event_cube128_traffic.json"]["files"])

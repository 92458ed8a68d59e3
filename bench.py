#!/usr/bin/env python
"""Benchmark: active-edge updates/s of the water-flow cycle on the 128^3 cube.

Workload (one "step"): the 3-D cube 128^3 (2,097,152 vertices, 6,242,304 edges), f1, f2
i.i.d. uniform integers in [1, 16] (uint8 SoA, seed 2), A = face x=0, B = face x=127,
solved for M = 400, 800 and 1600 (three full solves through the C ABI, each a complete
run of the cycle loop from initialisation to termination).  An active-edge update is
one live flow advanced by one cycle (the paper's Step 1 sweep).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is measured with inputs resident in HBM (CUDA events on
the solver's stream, L2 flushed before every timed step); ``e2e`` repeats the step
through the synchronous C-ABI call with host buffers (weights and sets copied in,
results copied out, all inside the timed region).  ``--impl reference`` times the CPU
oracle (the paper's cycle loop, single-threaded C) on a bounded sample of the same
workload.  With several GPUs (torchrun) every rank solves the same workload on its own
GPU (replicas; no data is exchanged) and the rank-0 line aggregates all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active-edge updates/s"
UNIT = "updates/s"
M_SWEEP = (400, 800, 1600)
WORKLOAD = {"workload": "cube3d_128_uniform16_faceA_x0_faceB_x127_M400_800_1600", "side": 128, "d": 3,
            "vertices": 128 ** 3, "edges": 3 * 128 * 128 * 127, "weights": "uint8 U{1..16}", "seed": 2,
            "M": list(M_SWEEP), "solves_per_step": 3, "l2": "flushed before every timed step (256 MiB write)"}
ORACLE_SAMPLE_CYCLES = 200      # cpu_baseline: first 200 cycles of the M=1600 solve
REFERENCE_STEP_CYCLES = 120     # --impl reference: first 120 cycles per step


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_rate(local_s: float, units_per_rank: float, world: int, device=None):
    """Whole-job (time, rate) over replicas: every rank processed ``units_per_rank`` units in
    ``local_s`` seconds; the job's time is the slowest rank's (max over ranks) and the units
    of all ranks add up.  With ``world`` > 1 the process group must be initialised (NCCL on
    GPUs; the tests use gloo on CPU)."""
    total_s = float(local_s)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return total_s, world * units_per_rank / total_s


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alg_bytes_of(slots: int, rec) -> int:
    """alg_bytes of a 16-int64 result record (updates, arrivals, improved, launched at 7, 13, 14, 8)."""
    return alg_bytes(slots, int(rec[7]), int(rec[13]), int(rec[14]), int(rec[8]))


def alg_bytes(slots: int, updates: int, arrivals: int, improved: int, launched: int) -> int:
    """Algorithmic bytes of a solve (the per-unit figures of the measurement plan): 8 B per
    active-edge update (read and write one remaining-time counter, Step 1), 13 B per arrival
    (quality, f2, the 8-byte offer), 6 B per edge slot of an improved vertex (f1, f2 and the
    neighbour's label) and 12 B per started flow."""
    return 8 * updates + 13 * arrivals + 6 * slots * improved + 12 * launched


def traffic_record(name: str):
    """A per-launch DRAM traffic record under profiles/ (ncu dram__bytes_read.sum +
    dram__bytes_write.sum), used only while the kernel sources it was taken from are unchanged."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            pj = json.load(f)
        if pj.get("kernel_source_sha256") == _kernel_sha(TRAFFIC[name]["files"]):
            return pj
    except Exception:
        pass
    return None


def roofline_block(alg: float, seconds: float, kernel: str, traffic=None, note: str = "") -> dict:
    """Roofline of a timed region: algorithmic bytes over its time against the measured HBM copy
    peak; with a matching ncu record, the DRAM bytes over the same time as well."""
    peak, src = peaks()
    gbs = alg / seconds / 1e9 if seconds > 0 else 0.0
    out = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "traffic": traffic, "peak_source": src, "kernel": kernel, "algorithmic_bytes": float(alg),
           "seconds": seconds}
    if traffic is not None and seconds > 0:
        out["dram_gbs"] = traffic / seconds / 1e9
        out["dram_frac"] = out["dram_gbs"] / peak
    if note:
        out["note"] = note
    return out


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(inst, max_cycles: int):
    """The oracle (O1, as it stands) on a bounded sample: the first cycles of the M=1600 solve."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 1600, max_cycles=max_cycles, trace=False,
                     allow_timeout=True)
    dt = time.perf_counter() - t0
    return {"value": r.updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {r.cycles} cycles of the M=1600 solve ({r.updates} updates, {dt:.1f} s, "
                      f"single-threaded C oracle O1)",
            "whole_step": whole_step_oracle()}


def whole_step_oracle():
    """The oracle's recorded time for the whole step (the three full 128^3 solves), from the run that
    wrote tests/golden/oracle_results.json on one x86 core: the early cycles a bounded sample times run
    from cache, so the whole step's rate is the fairer denominator."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_results.json")) as f:
            g = json.load(f)["cases"]
        sec = sum(g[f"cube3d_128_M{M}"]["oracle_seconds"] for M in M_SWEEP)
        upd = sum(g[f"cube3d_128_M{M}"]["updates"] for M in M_SWEEP)
        return {"seconds": sec, "updates": upd, "updates_per_s": upd / sec, "cores": 1,
                "where": "one x86 core of the build container (oracle_seconds in tests/golden/oracle_results.json)"}
    except Exception:
        return None


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1511_06441_gb300 import synth
    import oracle
    oracle.build()
    inst = synth.workload_cube(128, 1600)

    def step():
        t0 = time.perf_counter()
        r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 1600, max_cycles=REFERENCE_STEP_CYCLES,
                         trace=False, allow_timeout=True)
        return r.updates, time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        u, t = step()
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    sample = (f"each step = first {REFERENCE_STEP_CYCLES} cycles of the M=1600 solve of the 128^3 cube "
              f"({tot_u // max(args.steps, 1)} updates), single-threaded C oracle O1")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded SplitMix64)",
        "config": dict(WORKLOAD, parallelism="single CPU core"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "whole_step": whole_step_oracle()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1511_06441_gb300 import build, csp, synth
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()

    inst = synth.workload_cube(128, 1600)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    f1 = torch.from_numpy(inst.f1).to(dev)
    f2 = torch.from_numpy(inst.f2).to(dev)
    torch.cuda.synchronize()
    lat = csp.Lattice(inst.extents, f1, f2, stream=stream)
    lat.reserve(0)
    A = torch.from_numpy(inst.A).to(dev)
    B = torch.from_numpy(inst.B).to(dev)
    nM = len(M_SWEEP)
    rec = torch.zeros((nM, 16), dtype=torch.int64, device=dev)
    trace_cap = 4096
    trace = torch.zeros((nM, 3 * trace_cap), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    K, W = args.steps, args.warmup

    def step(evs=None):
        for i, M in enumerate(M_SWEEP):
            kb, ke = (evs[i] if evs else (None, None))
            lat.solve_async(A, B, M, rec[i], trace_dev=trace[i] if args.trace else None,
                            trace_cap=trace_cap if args.trace else 0, ctas=args.ctas, stream=stream,
                            ev_begin=kb, ev_end=ke)

    with torch.cuda.stream(stream):
        for _ in range(W):
            step()
        stream.synchronize()
        ref = rec.cpu().numpy().copy()
        if (ref[:, 0] != 0).any():
            raise RuntimeError(f"solve failed: status {ref[:, 0].tolist()}")
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        kern_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in M_SWEEP]
                   for _ in range(K)]
        for row in kern_ev:  # torch creates the CUDA event at its first record: do it now
            for a, b in row:
                a.record(stream)
                b.record(stream)
        sampler = ClockSampler(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.3)
        for k in range(K):
            flush.fill_(k & 0xFF)
            step_ev[k][0].record(stream)
            step(kern_ev[k])
            step_ev[k][1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if world > 1:
            torch.distributed.barrier()
    out = rec.cpu().numpy()
    assert (out[:, 0] == 0).all() and (out[:, 1:12] == ref[:, 1:12]).all(), "results changed between steps"
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    kern_ms = [[a.elapsed_time(b) for a, b in row] for row in kern_ev]
    upd_per_step = int(out[:, 7].sum())
    total_s, value = replica_rate(sum(step_ms) / 1e3, K * upd_per_step, world, dev)

    # roofline of the cycle kernel (the only kernel that scales with the work)
    d = 3
    alg_bytes = [alg_bytes_of(2 * d, r) for r in out]
    kern_avg_ms = float(np.mean(kern_ms))
    achieved = float(np.mean([alg_bytes[i] / (np.mean([kern_ms[k][i] for k in range(K)]) / 1e3) for i in range(nM)]))
    achieved /= 1e9
    peak, peak_src = peaks()
    traffic, dram = None, None
    pj = traffic_record("k_cycle_cube128_traffic.json")
    if pj is not None:
        per_m = pj["traffic_bytes_per_launch"]
        traffic = float(np.mean([per_m[str(M)] for M in M_SWEEP]))
        dram = dram_rate([per_m[str(M)] for M in M_SWEEP],
                         [float(np.mean([kern_ms[k][i] for k in range(K)])) for i in range(nM)])

    # end to end through the synchronous C-ABI call with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hf1 = torch.from_numpy(inst.f1).pin_memory()
        hf2 = torch.from_numpy(inst.f2).pin_memory()
        hA, hB = inst.A.copy(), inst.B.copy()
        lat2 = csp.Lattice(inst.extents, inst.f1, inst.f2)
        lat2.reserve(0)
        for _ in range(1):
            for M in M_SWEEP:
                lat2.solve(hA, hB, M, trace=args.trace, trace_cap=trace_cap)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e2e_upd = 0
        for _ in range(args.e2e_steps):
            lat2.upload_weights(hf1.numpy(), hf2.numpy())
            for M in M_SWEEP:
                r = lat2.solve(hA, hB, M, trace=args.trace, trace_cap=trace_cap)
                e2e_upd += r.updates
        torch.cuda.synchronize()
        dt, e2e_rate = replica_rate(time.perf_counter() - t0, e2e_upd, world, dev)
        h2d = inst.f1.nbytes + inst.f2.nbytes + nM * (hA.nbytes + hB.nbytes)
        d2h = nM * (16 * 8 + (3 * 8 * trace_cap if args.trace else 0))
        e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
               "ms_per_step": 1e3 * dt / args.e2e_steps}
        lat2.close()

    # the same three solves in the event form of the cycle loop (A/B against the sweep above)
    engines = None
    if args.engines and world == 1:
        engines = bench_engines(csp, lat, A, B, stream, trace, trace_cap, rec, out, kern_ms, args)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic (seeded SplitMix64 lattice weights)",
        "config": dict(WORKLOAD, parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       trace=bool(args.trace)),
        "results": {str(M): {"F1": int(r[1]), "X": int(r[2]), "x_src": int(r[3]), "x_dir": int(r[4]),
                             "F2": int(r[5]), "cycles": int(r[6]), "updates": int(r[7]), "passes": int(r[9]),
                             "max_pool": int(r[10]), "arrivals": int(r[13]), "improved": int(r[14]),
                             "launched": int(r[8]), "alg_bytes": alg_bytes[i],
                             "kernel_ms": float(np.mean([kern_ms[k][i] for k in range(K)]))}
                    for i, (M, r) in enumerate(zip(M_SWEEP, out))},
        "cube128_solves_per_s": world * K * nM / total_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "dram_gbs": dram, "dram_frac": dram / peak if dram is not None else None,
                     "kernel": "k_cycle (persistent cycle kernel)",
                     "algorithmic_bytes_per_launch": float(np.mean(alg_bytes)),
                     "kernel_ms_per_launch": kern_avg_ms},
        "gpu_launches": 4 * nM * K,
        "clocks": clocks,
        "e2e": e2e,
        "engines": engines,
        "shape": shape_info(csp),
    }
    del lat, f1, f2, flush, trace, rec
    torch.cuda.empty_cache()
    if world == 1 and args.batch:
        line["batched"] = bench_batched(csp, synth)
    if world == 1 and args.serve > 0:
        line["serving"] = bench_serving(csp, synth, args.serve, args.no_cpu_baseline,
                                        [float(x) for x in args.serve_rates.split(",")], bool(args.serve_plain))
    if world == 1 and args.anticorrelated:
        line["anticorrelated"] = bench_anticorrelated(csp, synth, args.no_cpu_baseline)
    if world == 1 and args.open_problems:
        line["open_problems"] = bench_open_problems(csp, synth)
    if world == 1 and args.fractal:
        line["fractal"] = bench_fractal(csp, synth)
    if world == 1 and args.graphs:
        line["graphs"] = bench_graphs(csp, synth, args.graph_side)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(inst, ORACLE_SAMPLE_CYCLES)
    line["summary"] = summary(line)  # last, so that a tail of the line keeps it
    print(json.dumps(line), flush=True)


def shape_info(csp) -> dict:
    """The block shape the library was built with and, if the shape tuner cached its choice, what it
    measured (paper_1511_06441_gb300/shape.json)."""
    out = {"built": csp.build_shape()}
    path = os.path.join(ROOT, "paper_1511_06441_gb300", "shape.json")
    if os.path.exists(path):
        with open(path) as f:
            t = json.load(f)
        out["tuner"] = {"chosen": t.get("chosen_label"), "gain_over_default": t.get("gain_over_default"),
                        "measured": [[m["shape"], m.get("cube128_step_ms"), m.get("batch512_ms", m.get("batch128_ms"))]
                                     for m in t.get("measured", [])]}
    return out


def summary(line: dict) -> dict:
    """The headline figures of every section, repeated compactly at the end of the line."""
    s = {"updates_per_s": line["value"], "roofline_frac": line["roofline"]["frac"],
         "e2e_updates_per_s": (line.get("e2e") or {}).get("value")}
    eng = line.get("engines")
    if eng:
        s["event_form_vs_sweep"] = eng.get("event_vs_sweep")
    b = line.get("batched")
    if b and "instances_per_s" in b:
        s["batched"] = {"instances_per_s": b["instances_per_s"], "plain_instances_per_s": b["plain_instances_per_s"],
                        "speedup_vs_plain": b["speedup_vs_plain"], "agree_with_plain": b["agree_with_plain"],
                        "roofline_frac": b["roofline"]["frac"]}
    v = line.get("serving")
    if v and v.get("rates"):
        s["serving"] = {"queries": v["queries"], "p99_ms_served_vs_plain": [
            [r["rate_x_saturation"], round(r["served"]["p99_ms"], 2), round(r["plain"]["p99_ms"], 2)] for r in v["rates"]],
            "served_p99_le_plain_everywhere": all(r["served"]["p99_ms"] <= r["plain"]["p99_ms"] for r in v["rates"]),
            "equal_to_alone": min(r["served"]["equal_to_alone"] for r in v["rates"])}
    a = line.get("anticorrelated")
    if a and "time_to_solution_s" in a:
        s["anticorrelated"] = {"time_to_solution_s": a["time_to_solution_s"], "answer_equals_oracle":
                               a["answer_equals_oracle"], "roofline_frac": a["roofline"]["frac"]}
    return s


def bench_engines(csp, lat, A, B, stream, trace, trace_cap, rec, sweep_out, sweep_ms, args):
    """The step's three solves in the event form (CSP_OPT_EVENT), kernel time by CUDA events on the
    solver's stream, one warm-up each; results must equal the sweep's."""
    import torch
    K = len(sweep_ms)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in M_SWEEP]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    ms = []
    with torch.cuda.stream(stream):
        for i, M in enumerate(M_SWEEP):
            for rep in range(2):
                lat.solve_async(A, B, M, rec[i], trace_dev=trace[i] if args.trace else None,
                                trace_cap=trace_cap if args.trace else 0, stream=stream, ev_begin=evs[i][0],
                                ev_end=evs[i][1], engine="event")
                stream.synchronize()
            ms.append(evs[i][0].elapsed_time(evs[i][1]))
    got = rec.cpu().numpy()
    same = bool((got[:, 1:9] == sweep_out[:, 1:9]).all())
    sweep_avg = [float(np.mean([sweep_ms[k][i] for k in range(K)])) for i in range(len(M_SWEEP))]
    upd = int(got[:, 7].sum())
    tr = traffic_record("k_event_cube128_traffic.json")
    ev_traffic = None
    if tr is not None:
        per_m = tr["traffic_bytes_per_launch"]
        ev_traffic = {"bytes_per_launch": [per_m[str(M)] for M in M_SWEEP],
                      "dram_gbs": dram_rate([per_m[str(M)] for M in M_SWEEP], ms)}
    return {"event_kernel_ms": ms, "sweep_kernel_ms": sweep_avg, "same_results": same, "event_dram": ev_traffic,
            "event_updates_per_s": upd / (sum(ms) / 1e3), "event_vs_sweep": sum(sweep_avg) / sum(ms),
            "default_form": lat.default_engine(),
            "note": "event form: per-edge queues and a calendar of arrival times (CSP_OPT_EVENT); the default "
                    "form for this lattice is the sweep (mean f1 8.5 < 64)"}


def bench_anticorrelated(csp, synth, no_cpu=False):
    """The 4096 x 4096 anti-correlated lattice (f1 geometric, f2 = 256 - f1, uint16, corner
    to corner, M = floor(1.2 F2*)): time to solution of one solve and the whole path from
    that solve (recorded first improvements + GPU backtrack), checked against the stored
    answer of the oracle's lexicographic Dijkstra (tests/golden/anticorrelated_lexmin.json)."""
    import torch
    side = 4096
    with open(os.path.join(ROOT, "tests", "golden", "anticorrelated_lexmin.json")) as f:
        g = json.load(f)["sides"][str(side)]
    inst = synth.workload_anticorrelated(side, M=g["M"])
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    lat.reserve(1 << 29)  # the flow pool peaks near 3.1e8 flows
    s = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for ev in (ev0, ev1):
        ev.record(s)  # (an event has a handle once recorded)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    path, r = lat.reconstruct_fast(inst.A, inst.B, inst.M, log_capacity=-1, time_limit_s=900, stream=s,
                                   ev_begin=ev0, ev_end=ev1)
    wall = time.perf_counter() - t0
    kern_s = ev0.elapsed_time(ev1) / 1e3
    # the path's own sums, read from the weight arrays
    st = synth.strides(inst.extents)
    V = inst.V
    f1 = inst.f1.reshape(-1).astype(np.int64)
    f2 = inst.f2.reshape(-1).astype(np.int64)
    a, b = path[:-1], path[1:]
    lo = np.minimum(a, b)
    k = np.where(np.abs(b - a) == st[0], 0, 1)
    adjacent = bool(np.isin(np.abs(b - a), st).all())
    sums = (int(f1[k * V + lo].sum()), int(f2[k * V + lo].sum())) if adjacent else (-1, -1)
    out = {
        "workload": "lattice2d_4096_anticorr_geom0.1_f2_256-f1_uint16_corner_to_corner_M1.2F2star",
        "M": inst.M, "F1": r.F1, "F2": r.F2, "X": r.X, "x": [r.x_src, r.x_dir],
        "answer_equals_oracle": r.answer() == (g["F1"], g["X"], g["x_src"], g["x_dir"], g["F2"]),
        "cycles": r.cycles, "updates": r.updates, "launched": r.launched, "improved": r.improved,
        "max_pool": r.max_pool,
        "time_to_solution_s": kern_s,
        "updates_per_s": r.updates / kern_s,
        "path_vertices": int(len(path)),
        "path_sums_equal_answer": sums == (r.F1, r.F2) and int(path[0]) == 0 and int(path[-1]) == r.X,
        "solve_and_path_wall_s": wall,
        "backtrack_and_copy_s": wall - kern_s,
        "note": "cycle kernel timed with CUDA events (first improvements recorded for the backtrack); "
                "the path needs one solve, repeated application would need one per path vertex",
    }
    tr = traffic_record("k_cycle_anticorr4096_traffic.json")
    out["roofline"] = roofline_block(alg_bytes(4, r.updates, r.arrivals, r.improved, r.launched), kern_s,
                                     "k_cycle (one persistent launch, the whole solve)",
                                     tr["traffic_bytes_per_launch"] if tr else None)
    lat.close()
    torch.cuda.empty_cache()
    if not no_cpu:
        out["cpu_baseline"] = cpu_baseline_anticorrelated(inst)
    return out


def cpu_baseline_anticorrelated(inst, cycles: int = 1500):
    """The oracle (O1, as it stands) on one core over a bounded sample of the 4096^2 solve: its first
    ``cycles`` cycles (the whole solve, 27,064 cycles with a pool of up to 3e8 flows, would take days)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, max_cycles=cycles, trace=False,
                     allow_timeout=True)
    dt = time.perf_counter() - t0
    return {"value": r.updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {r.cycles} cycles of the 4096^2 solve ({r.updates} updates, {dt:.1f} s, "
                      f"single-threaded C oracle O1); early cycles have small pools"}


def bench_open_problems(csp, synth, seeds=(6, 7, 8, 9), side=1024):
    """The paper's open problems (final section): the average size of the active set at time t,
    and the number of phantoms created, when travel times and weights are i.i.d. random.  2-D side x side lattices with
    f1 ~ U{1..16} and water from the centre vertex until it reaches a corner (or dies out);
    the per-cycle trace (active vertices, live flows) averaged over seeds at t = side/16 ..
    the end.  Three settings: f2 = 0 (travel times only, first-passage percolation: the
    setting of the paper's Lemma and Theorem), f2 ~ U{1..16} with a bound that never binds,
    and f2 ~ U{1..16} with M = 2 side (water dies out before the corners)."""
    out = {"workload": f"lattice2d_{side}_U16_point_source_B_corners", "seeds": list(seeds), "cases": []}
    for name, M, zero_f2 in (("f2 = 0", 1, True), ("f2 ~ U{1..16}, M never binds", (1 << 31) - 2, False),
                             (f"f2 ~ U{{1..16}}, M = {2 * side}", 2 * side, False)):
        traces, ph, la = [], [], []
        for seed in seeds:
            inst = synth.workload_point_source(side, seed)
            f2 = np.zeros_like(inst.f2) if zero_f2 else inst.f2
            lat = csp.Lattice(inst.extents, inst.f1, f2)
            r = lat.solve(inst.A, inst.B, M, trace=True, trace_cap=1 << 17, phantoms=True)
            traces.append(r.trace)
            ph.append(r.phantoms)
            la.append(r.launched)
            lat.close()
        t_end = min(int(tr[-1, 0]) for tr in traces)
        rows = []
        t = side // 16
        while t <= t_end:
            act, flo = [], []
            for tr in traces:
                k = int(np.searchsorted(tr[:, 0], t, side="right")) - 1  # the state at time t
                act.append(int(tr[k, 1]))
                flo.append(int(tr[k, 2]))
            ma = float(np.mean(act))
            rows.append({"t": t, "mean_active": ma, "active_per_t": ma / t,
                         "flows_per_active": float(np.sum(flo)) / max(1, float(np.sum(act)))})
            t *= 2
        out["cases"].append({"case": name, "M": M, "end_time_min_over_seeds": t_end, "rows": rows,
                             "mean_phantoms_per_solve": float(np.mean(ph)),
                             "phantoms_per_launched_flow": float(np.sum(ph)) / max(1, float(np.sum(la)))})
    return out


def bench_fractal(csp, synth, t=4096):
    """The environments omega_1 .. omega_k (t = 2^k) of the proof of the paper's t log t lower
    bound on the active set: N_t(omega_j), the active vertices at time t (all of V has
    |x| <= t), against the proof's N_t(omega_1) + (j - 1) 4t/15."""
    import torch
    k = t.bit_length() - 1
    rows = []
    for j in range(1, k + 1):
        inst = synth.fractal_environment(t, j)
        lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
        lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=t + 8)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=t + 8)
        sec = time.perf_counter() - t0
        lat.close()
        row = r.trace[int(np.searchsorted(r.trace[:, 0], t))]
        assert int(row[0]) == t
        rows.append({"j": j, "N_t": int(row[1]), "N_t_per_t": int(row[1]) / t, "live_flows": int(row[2]),
                     "F1": r.F1, "solve_ms": 1e3 * sec})
    n1 = rows[0]["N_t"]
    for x in rows:
        x["proof_N_t"] = n1 + (x["j"] - 1) * 4 * t / 15
    return {"workload": f"lattice2d_fractal_t{t}", "extents": [2 * t + 1, t + 2], "t": t, "rows": rows}


def bench_graphs(csp, synth, side=2048):
    """General graphs (csp_create_graph) against the lattice path: the 2-D side^2 lattice with
    f1, f2 ~ U{1..16} (seed 31) solved natively and written as a graph (the same solve, so the
    answers and counts must agree), and the king's graph of the same side (8 neighbours,
    seed 32).  A = column 0, B = the last column, M = 6 side.  Wall time of the synchronous
    call after one warm-up solve."""
    ext = [side, side]
    f1, f2 = synth.uniform_weights(ext, 1, 16, 31)
    A, B, M = synth.face(ext, 0, 0), synth.face(ext, 0, side - 1), 6 * side
    nbr, g1, g2 = synth.graph_from_lattice(ext, f1, f2)
    king = synth.king_graph(side, 1, 16, seed=32)
    out = {"workload": f"lattice2d_{side}_U16 native and as a graph; king{side}_U16", "M": M, "cases": []}
    ref = None
    for name, make, a, b in (("lattice (native)", lambda: csp.Lattice(ext, f1, f2), A, B),
                             ("lattice as a graph", lambda: csp.Graph(nbr, g1, g2), A, B),
                             ("king's graph", lambda: csp.Graph(king.nbr, king.f1, king.f2), king.A, king.B)):
        h = make()
        h.reserve()
        h.solve(a, b, M)
        t0 = time.perf_counter()
        r = h.solve(a, b, M)
        sec = time.perf_counter() - t0
        h.close()
        key = (r.answer(), r.cycles, r.updates, r.launched)
        if ref is None:
            ref = key
        out["cases"].append({"case": name, "answer": list(r.answer()), "cycles": r.cycles, "updates": r.updates,
                             "solve_s": sec, "updates_per_s": r.updates / sec,
                             "same_as_native": key == ref if name == "lattice as a graph" else None})
    return out


def bench_batched(csp, synth):
    """512 mixed 2-D/3-D instances: one tuned batched launch vs one launch per instance."""
    import torch
    insts = synth.batch_instances(512)
    lats = [csp.Lattice(i.extents, i.f1, i.f2) for i in insts]
    items = [(L, i.A, i.B, i.M) for L, i in zip(lats, insts)]
    b = csp.Batch(items)
    s = torch.cuda.Stream()

    def timed(run):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(s)
        run()
        ev[1].record(s)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1])

    b.run(s)  # warm-up with the first-guess schedule, then one autotuner step on its measurements
    torch.cuda.synchronize()
    res0 = b.results()
    b.tune(res0)
    ms_b = timed(lambda: b.run(s))
    res = b.results()
    model = b.model()
    sched = b.schedule()
    devA = [torch.from_numpy(i.A).cuda() for i in insts]
    devB = [torch.from_numpy(i.B).cuda() for i in insts]
    rec = torch.zeros((len(insts), 16), dtype=torch.int64, device="cuda")
    for L, i in zip(lats, insts):
        L.reserve()  # the default pool (with room for part-filled chunks); plain solves cannot grow it
    torch.cuda.synchronize()

    def plain():
        for k, (L, i) in enumerate(zip(lats, insts)):
            L.solve_async(devA[k], devB[k], i.M, rec[k], stream=s)

    ms_p = timed(plain)
    r = rec.cpu().numpy()
    agree = sum(1 for k in range(len(insts)) if r[k, 0] == 0 and tuple(int(x) for x in r[k, 1:6]) == res[k].answer())
    plain_ok = int((r[:, 0] == 0).sum())
    upd = sum(x.updates for x in res)
    try:
        cpu = cpu_baseline_batched(insts, [x.updates for x in res])
    except Exception as e:  # the GPU numbers stand without it
        cpu = {"error": f"{type(e).__name__}: {e}"}
    b.close()
    for L in lats:
        L.close()
    torch.cuda.empty_cache()
    n = len(insts)
    alg = sum(alg_bytes(2 * len(i.extents), x.updates, x.arrivals, x.improved, x.launched) for i, x in zip(insts, res))
    tr = traffic_record("k_batch_batch512_traffic.json")
    roof = roofline_block(alg, ms_b / 1e3, "k_batch (one persistent launch over all 512 instances)",
                          tr["traffic_bytes_per_launch"] if tr else None)
    return {"workload": "batch512_mixed_2d32-1024_3d16-160_U1-32_faceA_faceB", "instances": n,
            "roofline": roof,
            "instances_per_s": n / (ms_b / 1e3), "plain_instances_per_s": n / (ms_p / 1e3),
            "speedup_vs_plain": ms_p / ms_b, "batched_ms": ms_b, "plain_ms": ms_p,
            "updates_per_s": upd / (ms_b / 1e3), "updates": upd,
            "statuses_ok": sum(1 for x in res if x.status == 0), "plain_statuses_ok": plain_ok,
            "agree_with_plain": agree, "cpu_baseline": cpu,
            "schedule": {"ctas": sched["ctas"], "group_sizes": {str(g): int((sched["group"] == g).sum())
                                                                for g in sorted(set(sched["group"].tolist()))},
                         "planned_makespan_ms": model["makespan_us"] / 1e3,
                         "model": {k: round(v, 3) for k, v in model.items() if k != "makespan_us"}},
            "plain": "one cooperative launch per instance (csp_solve_async), sequential on one stream"}


def _oracle_updates(job):
    """One O1 solve in a worker process: returns its update count."""
    import oracle
    extents, f1, f2, A, B, M = job
    return oracle.cycle(extents, f1, f2, A, B, M, trace=False).updates


def cpu_baseline_batched(insts, updates, budget_updates=8e9, cap_updates=6e8, cores=None):
    """The oracle (O1, as it stands) over independent instances on all host cores: a bounded
    sample of the batch (every instance whose update count, known from the GPU run, is at most
    ``cap_updates``, in index order, until ``budget_updates`` are taken), one O1 per instance in
    a pool of spawned processes.  Reports instances/s on the sample and the whole batch's time
    estimated from the sample's updates/s (the same updates the GPU counted)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    pick, tot = [], 0
    for i, u in enumerate(updates):
        if u <= cap_updates and tot + u <= budget_updates:
            pick.append(i)
            tot += u
    jobs = [(insts[i].extents, insts[i].f1, insts[i].f2, insts[i].A, insts[i].B, insts[i].M) for i in pick]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        got = pool.map_async(_oracle_updates, jobs, chunksize=1).get(timeout=300)  # never wait forever
    wall = time.perf_counter() - t0
    if got != [updates[i] for i in pick]:
        raise RuntimeError("the oracle's update counts differ from the GPU's")
    rate = tot / wall
    est = float(sum(updates)) / rate
    return {"value": len(pick) / wall, "unit": "instances/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(pick)} of {len(insts)} instances (those with at most {cap_updates:.0e} updates, "
                      f"{tot:.3e} updates in all), one single-threaded O1 per instance over {cores} processes",
            "updates_per_s": rate, "whole_batch_estimate_s": est,
            "whole_batch_instances_per_s_estimate": len(insts) / est}


def bench_serving(csp, synth, n_queries, no_cpu=False, rates=None, plain=True):
    """48^4 lattice, query stream served with continuous batching vs answered one at a time."""
    import torch
    ext, f1, f2 = synth.serving_lattice(48, 4, 5)
    lat = csp.Lattice(ext, f1, f2)
    qs = synth.serving_queries(n_queries, ext, seed=5)
    t_svc = []
    alone = []
    for q in qs:
        t0 = time.perf_counter()
        alone.append(lat.solve(q.A, q.B, q.M))
        t_svc.append(time.perf_counter() - t0)
    mu = 1.0 / float(np.mean(t_svc))
    key = lambda r: (r.answer(), r.cycles, r.updates)  # noqa: E731
    max_pool = max(r.max_pool for r in alone)
    rates = tuple(rates or (0.25, 0.5, 0.75, 1.0, 1.25))
    out = {"workload": f"lattice4d_48_U1-20_{n_queries}queries_1-64src_hyperplaneB_M200-2000",
           "queries": n_queries, "plain_saturation_qps": mu, "service_ms_p50": 1e3 * float(np.median(t_svc)),
           "rates": []}
    srv = csp.Server(lat, group_ctas=16, wide_depth=3, pool_capacity=max(1 << 16, int(1.25 * max_pool)),
                     session_seconds=900)
    out["slots"] = srv.groups
    out["ctas_per_slot"] = srv.group_ctas
    out["modes"] = "the whole grid answers one query at a time while fewer than 3 wait; 16-CTA groups serve a " \
                   "backlog in parallel until all are idle (csp_server_options.wide_depth)"
    served = {}
    for m in rates:
        arr = synth.poisson_arrivals(n_queries, m * mu, seed=5)
        s0 = srv.stats()
        got, L, mk = srv.replay(qs, arr)
        s1 = srv.stats()
        served[m] = (got, L, mk, {k: s1[k] - s0[k] for k in s1})
    srv.close()
    alg = sum(alg_bytes(8, x.updates, x.arrivals, x.improved, x.launched) for x in alone)
    tr = traffic_record("k_server_lattice4d48_traffic.json")
    for m in rates:
        got, L, mk, modes = served[m]
        arr = synth.poisson_arrivals(n_queries, m * mu, seed=5)
        pg, PL, pmk = csp.plain_replay(lat, qs, arr) if plain else (None, np.full(1, np.nan), np.nan)
        out["rates"].append({
            "rate_x_saturation": m, "rate_qps": m * mu,
            "served": {"qps": n_queries / mk, "p50_ms": 1e3 * float(np.median(L)),
                       "p99_ms": 1e3 * float(np.quantile(L, 0.99)),
                       "equal_to_alone": sum(key(a) == key(b) for a, b in zip(got, alone)),
                       "answered_by": modes,
                       "roofline": roofline_block(alg, mk, "k_server (persistent, the whole stream)",
                                                  note="algorithmic bytes of all queries over the stream's makespan "
                                                       "(arrival-limited below saturation)")},
            "plain": {"qps": n_queries / pmk, "p50_ms": 1e3 * float(np.median(PL)),
                      "p99_ms": 1e3 * float(np.quantile(PL, 0.99))}})
    top = out["rates"][-1]["served"]["roofline"]
    out["roofline"] = dict(top, note="at the highest rate (1.25 x saturation: the server is busy throughout); "
                                     "per-rate blocks under rates[*].served.roofline",
                           traffic=tr["traffic_bytes_per_launch"] if tr else None)
    lat.close()
    torch.cuda.empty_cache()
    if not no_cpu:
        try:
            out["cpu_baseline"] = cpu_baseline_serving(n_queries, [x.updates for x in alone])
        except Exception as e:  # the GPU numbers stand without it
            out["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
    return out


_SERVE_STATE = {}


def _serve_init():
    from paper_1511_06441_gb300 import synth
    _SERVE_STATE["lat"] = synth.serving_lattice(48, 4, 5)


def _serve_oracle(job):
    """One O1 query on the 48^4 serving lattice in a worker process: returns its update count."""
    import oracle
    from paper_1511_06441_gb300 import synth
    ext, f1, f2 = _SERVE_STATE["lat"]
    q = synth.serving_queries(1, ext, seed=5, start=job)[0]
    return oracle.cycle(ext, f1, f2, q.A, q.B, q.M, trace=False).updates


def cpu_baseline_serving(n_queries, updates, budget_updates=6e9, cores=None):
    """The oracle (O1, as it stands) answering the query stream on all host cores: a bounded sample
    (the first queries in stream order until ``budget_updates`` updates, counts known from the GPU),
    one single-threaded O1 per query in a pool of spawned processes (each holds about 0.5 GB of
    per-vertex state).  Queries/s on the sample; no arrival process (as fast as the cores go)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    pick, tot = [], 0
    for i, u in enumerate(updates):
        if tot + u > budget_updates:
            break
        pick.append(i)
        tot += u
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores, initializer=_serve_init) as pool:
        got = pool.map_async(_serve_oracle, pick, chunksize=1).get(timeout=300)
    wall = time.perf_counter() - t0
    if got != [updates[i] for i in pick]:
        raise RuntimeError("the oracle's update counts differ from the GPU's")
    return {"value": len(pick) / wall, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {len(pick)} of {n_queries} queries ({tot:.3e} updates), one single-threaded O1 "
                      f"per query over {cores} processes, no arrival process",
            "updates_per_s": tot / wall}


def dram_rate(traffic_bytes, kernel_ms):
    """DRAM GB/s of the cycle kernel: per launch, the ncu DRAM bytes (read + write) of that
    solve over its CUDA-event time, averaged over the solves of a step."""
    if len(traffic_bytes) != len(kernel_ms) or not kernel_ms:
        raise ValueError("one traffic figure per timed solve")
    return float(np.mean([b / (ms / 1e3) for b, ms in zip(traffic_bytes, kernel_ms)])) / 1e9


# Per-launch DRAM traffic records under profiles/: the sources each kernel is built from (a record
# counts only while they are unchanged), the launch labels, and which captured launches they take.
TRAFFIC = {
    "k_cycle_cube128_traffic.json": {"files": ("csp_device.cuh", "csp_solver.cu"), "labels": ["400", "800", "1600"],
                                     "take": [0, 1, 2], "kernel": "k_cycle<3, uint8, trace=1> (128^3 cube)"},
    "k_event_cube128_traffic.json": {"files": ("csp_device.cuh", "csp_event.cuh", "csp_event.cu"),
                                     "labels": ["400", "800", "1600"], "take": [1, 3, 5],
                                     "kernel": "k_event<3, uint8, trace=1> (128^3 cube, second of two launches per M)"},
    "k_batch_batch512_traffic.json": {"files": ("csp_device.cuh", "csp_batch.cu"), "labels": None, "take": [0],
                                      "kernel": "k_batch<uint8> (512 mixed instances, tuned schedule)"},
    "k_server_lattice4d48_traffic.json": {"files": ("csp_device.cuh", "csp_server.cu"), "labels": None, "take": [0],
                                          "kernel": "k_server<4, uint8> (48^4 lattice, the whole session)"},
    "k_cycle_anticorr4096_traffic.json": {"files": ("csp_device.cuh", "csp_solver.cu"), "labels": None, "take": [0],
                                          "kernel": "k_cycle<2, uint16, trace=0> (4096^2 anti-correlated, the whole solve)"},
}


def _kernel_sha(files=("csp_device.cuh", "csp_solver.cu")):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1511_06441_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def record_traffic(csv_path: str, name: str, command: str, out_dir: str = "") -> dict:
    """Writes profiles/<name> from an ncu CSV (--metrics dram__bytes_read.sum,dram__bytes_write.sum,
    gpu__time_duration.sum --csv --print-units base): per captured launch, DRAM read + write bytes."""
    import csv
    spec = TRAFFIC[name]
    launches = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if len(r) > 5]
    head = rows[0]
    col = {k: head.index(k) for k in ("ID", "Metric Name", "Metric Value")}
    for r in rows[1:]:
        if not r[col["ID"]].isdigit():
            continue
        d = launches.setdefault(int(r[col["ID"]]), {})
        d[r[col["Metric Name"]]] = float(r[col["Metric Value"]].replace(",", ""))
    ids = sorted(launches)
    picked = [launches[ids[i]] for i in spec["take"]]
    traffic = [x["dram__bytes_read.sum"] + x["dram__bytes_write.sum"] for x in picked]
    dur = [x["gpu__time_duration.sum"] for x in picked]
    rec = {"kernel": spec["kernel"], "command": command, "kernel_sources": list(spec["files"]),
           "kernel_source_sha256": _kernel_sha(spec["files"])}
    if spec["labels"]:
        rec["traffic_bytes_per_launch"] = dict(zip(spec["labels"], traffic))
        rec["duration_ns_under_ncu"] = dict(zip(spec["labels"], dur))
    else:
        rec["traffic_bytes_per_launch"] = traffic[0]
        rec["duration_ns_under_ncu"] = dur[0]
    with open(os.path.join(out_dir or os.path.join(ROOT, "profiles"), name), "w") as f:
        json.dump(rec, f, indent=1)
    return rec


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--trace", type=int, default=1, help="record the per-cycle trace (active set size) in the step")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--engines", type=int, default=1, help="also time the step's solves in the event form (N=1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=1, help="also measure 512 batched instances vs one launch each (N=1)")
    ap.add_argument("--open-problems", type=int, default=0,
                    help="also measure the mean active-set size vs time on 1024^2 i.i.d. lattices (N=1)")
    ap.add_argument("--graphs", type=int, default=0,
                    help="also time general graphs against the lattice path on 2048^2 (N=1)")
    ap.add_argument("--graph-side", type=int, default=2048, help="side of the --graphs lattices")
    ap.add_argument("--fractal", type=int, default=0,
                    help="also count the active vertices at time t = 4096 on the environments omega_j (N=1)")
    ap.add_argument("--anticorrelated", type=int, default=1,
                    help="also time the 4096^2 anti-correlated solve and its path (N=1; ~1.5 min)")
    ap.add_argument("--serve-rates", default="0.25,0.5,0.75,1.0,1.25",
                    help="serving rates as multiples of the plain solver's saturation rate")
    ap.add_argument("--serve-plain", type=int, default=1, help="also replay the stream one query at a time")
    ap.add_argument("--serve", type=int, default=10000,
                    help="queries per rate for the serving comparison on the 48^4 lattice (0 = skip; N=1 only)")
    ap.add_argument("--record-traffic", nargs=3, metavar=("NCU_CSV", "NAME", "COMMAND"),
                    help="write profiles/NAME (a per-launch DRAM traffic record) from an ncu CSV and exit")
    args = ap.parse_args()
    if args.record_traffic:
        csv_path, name, command = args.record_traffic
        print(json.dumps(record_traffic(csv_path, name, command)))
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

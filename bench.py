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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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
                      f"single-threaded C oracle O1)"}


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
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    upd_per_step = int(out[:, 7].sum())
    value = world * K * upd_per_step / total_s

    # roofline of the cycle kernel (the only kernel that scales with the work)
    d = 3
    alg_bytes = [8 * int(r[7]) + 13 * int(r[13]) + 2 * d * 6 * int(r[14]) + 12 * int(r[8]) for r in out]
    kern_avg_ms = float(np.mean(kern_ms))
    achieved = float(np.mean([alg_bytes[i] / (np.mean([kern_ms[k][i] for k in range(K)]) / 1e3) for i in range(nM)]))
    achieved /= 1e9
    peak, peak_src = peaks()
    traffic = None
    prof = os.path.join(ROOT, "profiles", "k_cycle_cube128_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                pj = json.load(f)
            if pj.get("kernel_source_sha256") == _kernel_sha():
                traffic = pj.get("traffic_bytes_per_launch")
        except Exception:
            traffic = None

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
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        h2d = inst.f1.nbytes + inst.f2.nbytes + nM * (hA.nbytes + hB.nbytes)
        d2h = nM * (16 * 8 + (3 * 8 * trace_cap if args.trace else 0))
        e2e = {"value": world * e2e_upd / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
               "ms_per_step": 1e3 * dt / args.e2e_steps}
        lat2.close()

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
                             "max_pool": int(r[10]), "kernel_ms": float(np.mean([kern_ms[k][i] for k in range(K)]))}
                    for i, (M, r) in enumerate(zip(M_SWEEP, out))},
        "instances_per_s": world * K * nM / total_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": "k_cycle (persistent cycle kernel)",
                     "algorithmic_bytes_per_launch": float(np.mean(alg_bytes)),
                     "kernel_ms_per_launch": kern_avg_ms},
        "gpu_launches": 5 * nM * K,
        "clocks": clocks,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(inst, ORACLE_SAMPLE_CYCLES)
    print(json.dumps(line), flush=True)


def _kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("csp_device.cuh", "csp_solver.cu"):
        with open(os.path.join(ROOT, "paper_1511_06441_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--trace", type=int, default=1, help="record the per-cycle trace (active set size) in the step")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

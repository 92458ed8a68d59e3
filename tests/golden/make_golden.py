"""Writes oracle_results.json: O1 results, traces and label digests for the full-size
workloads, so GPU parity tests at those sizes need not rerun the (minutes-long) oracle.

Calls only the oracle (``oracle/``) and the seeded input generator.  Each entry records
a SHA-256 of the generated weights so that a change of the generator is detected.

    python tests/golden/make_golden.py            # all cases (~5 min)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1511_06441_gb300 import synth  # noqa: E402


def digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def case(inst, M):
    t0 = time.time()
    r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True)
    return {
        "extents": list(inst.extents), "M": M,
        "weights_sha256": digest(inst.f1, inst.f2),
        "result": [r.F1, r.X, r.x_src, r.x_dir, r.F2],
        "cycles": r.cycles, "updates": r.updates, "launched": r.launched,
        "trace": r.trace.tolist(),
        "labels_sha256": digest(r.labels.astype(np.int32)),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def main():
    out = {"generator": "paper_1511_06441_gb300.synth", "oracle": "oracle.cycle (O1)", "cases": {}}
    c1 = synth.workload_64x64()
    for M in (200, 250, 300, 400):
        out["cases"][f"lattice2d_64x64_M{M}"] = case(c1, M)
    c2 = synth.workload_cube(128, 1600)
    for M in (400, 800, 1600):
        out["cases"][f"cube3d_128_M{M}"] = case(c2, M)
        print(M, out["cases"][f"cube3d_128_M{M}"]["result"], flush=True)
    with open(os.path.join(HERE, "oracle_results.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()

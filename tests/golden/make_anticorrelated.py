"""Writes anticorrelated_lexmin.json: for the anti-correlated 2-D workload (f1 geometric
with p = 0.1 clipped to [1, 255], f2 = 256 - f1, A and B opposite corners, seed 3) at each
side, the lexicographically smallest (F1, F2) walk from the oracle's Dijkstra, its end X
and last edge x, and the bound M = floor(1.2 F2) the workload is run with.  Since F2 < M,
(F1, F2, X, x) is also the answer of a solve with that bound (Section 1), so GPU tests
and the benchmark use it at the full 4096 x 4096 size, where the cycle oracle would run
for days.

Calls only the oracle (``oracle/``) and the seeded input generator.  Each entry records
a SHA-256 of the generated weights so that a change of the generator is detected.

    python tests/golden/make_anticorrelated.py      # ~20 s
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1511_06441_gb300 import synth  # noqa: E402

SIDES = (128, 256, 512, 1024, 2048, 4096)
SEED = 3


def main():
    out = {"workload": "lattice2d anti-correlated: f1 = min(255, Geometric(0.1)), f2 = 256 - f1 (uint16), "
                       "A = {corner 0}, B = {opposite corner}, M = floor(1.2 F2*)",
           "seed": SEED, "sides": {}}
    for side in SIDES:
        inst = synth.workload_anticorrelated(side, seed=SEED)
        F1, F2, X, xs, xd = oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, full=True)
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(inst.f1).tobytes())
        h.update(np.ascontiguousarray(inst.f2).tobytes())
        out["sides"][str(side)] = {"F1": F1, "F2": F2, "X": X, "x_src": xs, "x_dir": xd,
                                   "M": (12 * F2) // 10, "weights_sha256": h.hexdigest()}
        print(side, out["sides"][str(side)], flush=True)
    with open(os.path.join(HERE, "anticorrelated_lexmin.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

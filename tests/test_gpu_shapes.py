"""Every block shape gives the same results: the library built with another shape (256
threads x 4 flows per tile, so a 1024-flow pool chunk instead of 2048; 4 CTAs per SM)
solves the tuning workloads (the 128^3 cube for M = 400, 800, 1600 with a trace, and the
512 mixed instances in one batched launch) with exactly the answers and counts of the
default build.  Each build runs in a process of its own, as the shape tuner runs them."""
import json
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _measure(lib):
    p = subprocess.run([sys.executable, "-m", "paper_1511_06441_gb300.tune", "--measure", lib], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_another_shape_gives_the_default_results():
    from paper_1511_06441_gb300 import build
    default = _measure(build.build())
    other_shape = {"tpb": 256, "ipt": 4, "nstage": 3, "min_ctas_per_sm": 4, "batch_min_ctas_per_sm": 2}
    lib = build.build(force=True, shape=other_shape, out=os.path.join(tempfile.mkdtemp(), "libcsp_other.so"))
    other = _measure(lib)
    assert other["shape"] == other_shape and default["shape"] != other_shape
    assert len(default["results"]) == 3 + 512
    assert other["results"] == default["results"]
    assert all(r[-1] == 0 for r in default["results"][3:])  # every batched instance solved

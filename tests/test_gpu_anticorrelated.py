"""The anti-correlated 2-D workload on the GPU: f1 = min(255, Geometric(0.1)), f2 = 256 - f1
(uint16), A and B opposite corners, M = floor(1.2 F2*) with F2* the weight of the
lexicographically smallest (F1, F2) walk.

* 128 x 128: the whole result (answer, cycles, updates, launched, per-cycle trace, labels)
  against the cycle oracle O1;
* 512 x 512 and the full 4096 x 4096: (F1, F2, X, x) against the oracle's lexicographic
  Dijkstra (tests/golden/anticorrelated_lexmin.json, written by make_anticorrelated.py).
  Since F2* < M the bound does not bind and that walk is the answer (Section 1);
* 4096 x 4096, first 1500 cycles: trace rows, updates and launched flows against O1 run
  for the same number of cycles; at 512 x 512 the trace against the solve's own counts;
* 48 x 48: the reconstructed path against the oracle's repeated application; 128 x 128:
  the path's adjacency and sums; 4096 x 4096: the whole path from one recorded solve
  against the oracle Dijkstra's predecessor chain.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1511_06441_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "anticorrelated_lexmin.json")


@pytest.fixture(scope="module")
def csp():
    from paper_1511_06441_gb300 import build, csp as mod
    build.build()
    return mod


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)["sides"]


def _instance(side, golden):
    inst = synth.workload_anticorrelated(side, M=golden[str(side)]["M"])
    return inst


def test_128_whole_result_equals_cycle_oracle(csp, golden):
    inst = _instance(128, golden)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=4096, phantoms=True)
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched, got.phantoms) == (want.cycles, want.updates, want.launched,
                                                                     want.phantoms)
    np.testing.assert_array_equal(got.trace, want.trace)
    np.testing.assert_array_equal(lat.labels(), want.labels.astype(np.int32))
    g = golden["128"]
    assert got.answer() == (g["F1"], g["X"], g["x_src"], g["x_dir"], g["F2"])
    lat.close()


@pytest.mark.parametrize("side", [256, 512])
def test_answer_equals_lexicographic_dijkstra(csp, golden, side):
    inst = _instance(side, golden)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, inst.M)
    g = golden[str(side)]
    assert got.answer() == (g["F1"], g["X"], g["x_src"], g["x_dir"], g["F2"])
    lat.close()


@pytest.fixture(scope="module")
def full(csp, golden):
    inst = _instance(4096, golden)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    lat.reserve(1 << 29)  # the pool peaks near 3.1e8 flows
    yield inst, lat
    lat.close()


def test_full_size_first_cycles_equal_cycle_oracle(csp, full):
    inst, lat = full
    K = 1500
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, max_cycles=K, allow_timeout=True)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=K + 8, max_cycles=K, check=False)
    assert got.status == csp.ERR_TIMEOUT and got.cycles == K == want.cycles
    assert (got.updates, got.launched) == (want.updates, want.launched)
    np.testing.assert_array_equal(got.trace[:K], want.trace[:K])


def test_full_size_answer_equals_lexicographic_dijkstra(csp, golden, full):
    inst, lat = full
    got = lat.solve(inst.A, inst.B, inst.M, time_limit_s=900)
    g = golden["4096"]
    assert got.answer() == (g["F1"], g["X"], g["x_src"], g["x_dir"], g["F2"])
    assert got.cycles <= got.F1 and got.launched >= got.improved >= got.cycles
    assert lat.labels()[got.X] == inst.M - got.F2


def test_full_size_path_equals_lexicographic_dijkstra(csp, golden, full):
    """The whole 4096 x 4096 path from one recorded solve and a GPU backtrack (first
    improvements only: the bound does not bind, so every path vertex is reached at its
    first improvement) against the oracle Dijkstra's predecessor chain, which is the path
    repeated application finds here (pinned in tests/test_oracle_pins.py)."""
    inst, lat = full
    F1, F2, X, xs, xd, want = oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, path=True)
    got, r = lat.reconstruct_fast(inst.A, inst.B, inst.M, log_capacity=-1, time_limit_s=900)
    assert r.answer() == (F1, X, xs, xd, F2)
    assert got.tolist() == want
    assert _path_sums(inst, want) == (F1, F2)


def test_trace_counts_add_up_to_updates(csp, golden):
    inst = _instance(512, golden)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=1 << 14)
    tr = got.trace
    assert len(tr) == got.cycles + 1 and tr[0, 0] == 0 and tr[-1, 0] == got.F1
    assert (np.diff(tr[:, 0]) > 0).all() and (tr[:, 1:] >= 0).all()
    assert int(tr[: got.cycles, 2].sum()) == got.updates  # flows alive at each cycle start
    lat.close()


def _path_sums(inst, path):
    st = synth.strides(inst.extents)
    V = inst.V
    f1 = inst.f1.reshape(-1).astype(np.int64)
    f2 = inst.f2.reshape(-1).astype(np.int64)
    t = w = 0
    for a, b in zip(path, path[1:]):
        lo, diff = min(a, b), abs(b - a)
        k = max(i for i, sk in enumerate(st) if sk == diff and inst.extents[i] > 1)  # (extent-1 axes repeat a stride)
        c = synth.coords(np.array([lo]), inst.extents)[0]
        assert c[k] + 1 < inst.extents[k] and f1[k * V + lo] > 0, (a, b)
        t += f1[k * V + lo]
        w += f2[k * V + lo]
    return int(t), int(w)


def test_48_path_equals_repeated_application_oracle(csp):
    F1, F2, _, _, _ = oracle.lexmin([48, 48], *synth.anticorrelated_weights([48, 48]), [0], [48 * 48 - 1],
                                    full=True)
    inst = synth.workload_anticorrelated(48, M=(12 * F2) // 10)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    r = lat.solve(inst.A, inst.B, inst.M)
    got = lat.reconstruct(inst.A, inst.B, inst.M, result=r)
    assert got.tolist() == want
    assert _path_sums(inst, want) == (r.F1, r.F2) == (F1, F2)
    lat.close()


def test_128_path_invariants(csp, golden):
    inst = _instance(128, golden)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    r = lat.solve(inst.A, inst.B, inst.M)
    path = lat.reconstruct(inst.A, inst.B, inst.M, result=r)
    assert path[0] == 0 and path[-1] == r.X == inst.V - 1
    assert len(set(path.tolist())) == len(path)
    assert _path_sums(inst, path.tolist()) == (r.F1, r.F2)
    lat.close()

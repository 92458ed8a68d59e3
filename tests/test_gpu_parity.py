"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

All results are integers and must match exactly: F1, X, x, F2, the cycle count, the
active-edge update count, the number of flows started, the per-cycle trace (Time,
active vertices, live flows), the phantom count and the final label array.

Sizes: tiny random lattices (1 CTA and several CTAs, so every barrier and compaction
path runs on ragged tails), medium lattices spanning many 2048-flow tiles, the 64x64
workload, and the full 128^3 cube against stored oracle results
(tests/golden/oracle_results.json, written by tests/golden/make_golden.py).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_results.json")


@pytest.fixture(scope="module")
def csp():
    from paper_1511_06441_gb300 import build, csp as mod
    build.build()
    return mod


def _check_same(lat, got, want, trace=True, labels=True):
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched) == (want.cycles, want.updates, want.launched)
    if trace:
        np.testing.assert_array_equal(got.trace, want.trace)
        if got.phantoms >= 0:  # counted when requested (trace mode)
            assert got.phantoms == want.phantoms
    if labels:
        np.testing.assert_array_equal(lat.labels(), want.labels.astype(np.int32))


def _run_pair(csp, inst, ctas=0, M=None, **kw):
    M = inst.M if M is None else M
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, M, trace=True, ctas=ctas, phantoms=True, **kw)
    _check_same(lat, got, want)
    lat.close()
    return got, want


@pytest.mark.parametrize("seed", range(0, 120))
def test_tiny_one_cta(csp, seed):
    _run_pair(csp, synth.random_small_instance(seed, max_vertices=24, dims=(1, 2, 3, 4)), ctas=1)


@pytest.mark.parametrize("seed", range(500, 560))
def test_tiny_several_ctas(csp, seed):
    inst = synth.random_small_instance(seed, max_vertices=40, f_lo=(0, 1), f_hi=9)
    inst.M = 30 + seed % 40
    _run_pair(csp, inst, ctas=1 + seed % 7)


MEDIUM = [
    ([100, 80], 1, 12, 0, 120, np.uint8),
    ([100, 80], 1, 12, 0, 400, np.uint8),
    ([24, 24, 24], 1, 16, 0, 160, np.uint8),
    ([24, 24, 24], 1, 16, 1, 90, np.uint8),
    ([9, 9, 9, 9], 1, 20, 0, 200, np.uint8),
    ([300, 7], 1, 300, 0, 5000, np.uint16),
    ([2000], 1, 40, 0, 100000, np.uint16),
]


@pytest.mark.parametrize("case", range(len(MEDIUM)))
@pytest.mark.parametrize("ctas", [0, 3, 64])
def test_medium(csp, case, ctas):
    ext, lo, hi, faces, M, dt = MEDIUM[case]
    f1, f2 = synth.uniform_weights(ext, lo, hi, 40 + case, dtype=dt)
    holes = synth.uniform_unit(40 + case, 9, f1.size).reshape(f1.shape) < 0.05
    f1[holes] = 0
    f2[holes] = 0
    if faces == 0:
        A, B = synth.face(ext, 0, 0), synth.face(ext, 0, ext[0] - 1)
    else:  # a few random sources, a random target set
        V = synth.num_vertices(ext)
        A = np.unique(synth.uniform_int(case, 3, 6, 0, V - 1))
        B = np.setdiff1d(np.unique(synth.uniform_int(case, 4, 50, 0, V - 1)), A)
    _run_pair(csp, synth.Instance(ext, f1, f2, A, B, M), ctas=ctas)


@pytest.mark.parametrize("M", [200, 250, 300, 400])
def test_lattice_64x64(csp, M):
    inst = synth.workload_64x64()
    got, want = _run_pair(csp, inst, M=M)
    if M == 200:
        assert got.F1 == -1  # no path across with F2 < 200 (the minimum F2 is 230)


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def cube(csp):
    inst = synth.workload_cube(128, 1600)
    g = json.load(open(GOLDEN))["cases"]
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    yield inst, lat, g
    lat.close()


@pytest.mark.parametrize("M", [400, 800, 1600])
def test_cube128_full_size_against_stored_oracle(csp, cube, M):
    inst, lat, g = cube
    want = g[f"cube3d_128_M{M}"]
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(inst.f1).tobytes())
    h.update(np.ascontiguousarray(inst.f2).tobytes())
    assert h.hexdigest() == want["weights_sha256"], "input generator changed: rerun tests/golden/make_golden.py"
    got = lat.solve(inst.A, inst.B, M, trace=True, trace_cap=4096)
    assert list(got.answer()) == want["result"]
    assert (got.cycles, got.updates, got.launched) == (want["cycles"], want["updates"], want["launched"])
    np.testing.assert_array_equal(got.trace, np.array(want["trace"], dtype=np.int64))
    assert _digest(lat.labels()) == want["labels_sha256"]
    # the untraced solve (the benchmark's configuration) gives the same answer and counts
    fast = lat.solve(inst.A, inst.B, M)
    assert fast.answer() == got.answer()
    assert (fast.cycles, fast.updates, fast.launched) == (got.cycles, got.updates, got.launched)
    assert _digest(lat.labels()) == want["labels_sha256"]


@pytest.mark.parametrize("ctas", [1, 37, 150, 304])
def test_cube128_independent_of_grid_size(csp, cube, ctas):
    inst, lat, g = cube
    want = g["cube3d_128_M800"]
    got = lat.solve(inst.A, inst.B, 800, ctas=ctas)
    assert list(got.answer()) == want["result"]
    assert (got.cycles, got.updates) == (want["cycles"], want["updates"])


@pytest.mark.parametrize("ext", [[1024, 1024], [96, 96, 96]])
def test_f2_zero_first_passage_at_size(csp, ext):
    # f2 = 0: F1 and the whole trace follow from plain Dijkstra (scipy), at any size
    f1, _ = synth.uniform_weights(ext, 1, 9, 21)
    f2 = np.zeros_like(f1)
    V = synth.num_vertices(ext)
    A = np.unique(synth.uniform_int(21, 3, 4, 0, V - 1))
    B = np.setdiff1d(synth.face(ext, 1, ext[1] - 1), A)
    F1, X, tau, rows = brute.dijkstra_trace(ext, f1, A, B)
    lat = csp.Lattice(ext, f1, f2)
    M = 2**31 - 2  # the largest bound the solver accepts (2^31 - 1 marks removed vertices)
    got = lat.solve(A, B, M, trace=True, trace_cap=1 << 15)
    assert (got.F1, got.X, got.F2) == (F1, X, 0)
    np.testing.assert_array_equal(got.trace, rows)
    lab = lat.labels()
    reached = np.isfinite(tau) & (tau <= F1)
    assert (lab[reached] == M).all() and (lab[~reached] == 0).all()
    lat.close()


@pytest.mark.parametrize("M", [2**31 - 2, 2**20, 140000])
def test_both_pool_formats(csp, M):
    # A path of 16,512 vertices with travel times up to 40,000 (16-bit weights).  With
    # M = 2^31 - 2 the flow word (18 bits), the quality (31 bits) and the arrival time (16
    # bits) do not fit one 64-bit word and the pool keeps three arrays; with M = 2^20 they
    # fit and each flow is one packed word.  Arrival times reach 3.3e8, far beyond the
    # 16-bit time field of the packed form; at M = 140,000 the only path is too heavy.
    ext = [16512]
    f1, f2 = synth.uniform_weights(ext, 1, 40000, 123, dtype=np.uint16)
    f2 = (f2 % 16 + 1).astype(np.uint16)
    assert int(f1[:16511].max()) >= 1 << 15
    inst = synth.Instance(ext, f1, f2, np.array([0], np.int64), np.array([16511], np.int64), M, "path16512")
    got, want = _run_pair(csp, inst)
    assert (got.F1 == -1) == (M == 140000)


def test_edge_cases(csp):
    ext = [6, 5]
    f1, f2 = synth.uniform_weights(ext, 1, 5, 3)
    lat = csp.Lattice(ext, f1, f2)
    # M <= 0: infeasible, one trace row
    r = lat.solve([0], [29], 0, trace=True)
    assert r.F1 == -1 and r.cycles == 0 and r.trace.tolist() == [[0, 0, 0]]
    # duplicates are sets
    a = lat.solve([0, 0, 1, 1], [29, 29], 40, trace=True)
    b = lat.solve([1, 0], [29], 40, trace=True)
    assert a.answer() == b.answer() and (a.trace == b.trace).all()
    # invalid: overlap, out of range, empty, M too large
    for A, B, M in (([0, 1], [1], 10), ([0], [30], 10), ([], [3], 10), ([0], [3], 2**31)):
        with pytest.raises(csp.CspError) as e:
            lat.solve(A, B, M)
        assert e.value.status == csp.ERR_INVALID
    # a source with no edges at all
    g1, g2 = f1.copy(), f2.copy()
    g1[0, 0] = g1[1, 0] = 0
    iso = csp.Lattice(ext, g1, g2)
    r = iso.solve([0], [29], 100, trace=True)
    assert r.F1 == -1 and r.trace.tolist() == [[0, 0, 0]]
    # A next to B: one cycle
    r = lat.solve([0], [1], 100)
    assert r.F1 == int(f1[0, 0]) and r.cycles == 1
    lat.close()
    iso.close()


def test_pool_growth_and_cycle_limit(csp):
    inst = synth.workload_cube(24, 300)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 300)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, 300, pool_capacity=100, trace=True)  # doubles until it fits
    assert got.answer() == want.answer() and (got.trace == want.trace).all()
    r = lat.solve(inst.A, inst.B, 300, max_cycles=5, check=False)
    assert r.status == csp.ERR_TIMEOUT and r.cycles == 5
    lat.close()


def test_async_device_resident(csp):
    torch = pytest.importorskip("torch")
    inst = synth.workload_cube(40, 500)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 500)
    lat = csp.Lattice(inst.extents, torch.from_numpy(inst.f1).cuda(), torch.from_numpy(inst.f2).cuda())
    lat.reserve()
    A = torch.from_numpy(inst.A).cuda()
    B = torch.from_numpy(inst.B).cuda()
    rec = torch.zeros(16, dtype=torch.int64, device="cuda")
    tr = torch.zeros(3 * 4096, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    for _ in range(2):  # twice: the workspace is reused
        lat.solve_async(A, B, 500, rec, trace_dev=tr, trace_cap=4096, stream=s)
        s.synchronize()
        r = csp.result_from_record(rec.cpu().numpy())
        assert r.status == csp.OK and r.answer() == want.answer()
        n = int(rec[11].item())
        np.testing.assert_array_equal(tr[: 3 * n].view(-1, 3).cpu().numpy(), want.trace)
    # invalid ids are reported in the record
    bad = torch.tensor([inst.A[0]], dtype=torch.int64, device="cuda")
    lat.solve_async(bad, bad, 500, rec, stream=s)
    s.synchronize()
    assert int(rec[0].item()) == csp.ERR_INVALID
    lat.close()

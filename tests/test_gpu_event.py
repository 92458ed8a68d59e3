"""GPU parity of the event-driven form (CSP_OPT_EVENT: a calendar of arrival times and
per-edge queues of flows in flight) against the CPU oracle, element by element: F1, X, x,
F2, cycles, active-edge updates, flows started, the per-cycle trace (Time, active vertices,
live flows), phantoms and the final labels.  Integer results: the tolerance is zero.

Sizes and shapes follow the sweep form's parity tests: tiny lattices of dimension 1-4 on
one CTA and on several (ragged tails, every barrier and claim path), medium lattices whose
calendar spans many chunks (8- and 16-bit weights, absent edges), the 64x64 workload, the
full 128^3 cube against the stored oracle results, f2 = 0 against plain Dijkstra at size,
general graphs and digraphs, fast reconstruction against repeated application, a window of
W = 512 (the largest the form takes) and the degenerate cases.
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


def _check_same(lat, got, want, labels=True):
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched) == (want.cycles, want.updates, want.launched)
    np.testing.assert_array_equal(got.trace, want.trace)
    if got.phantoms >= 0:
        assert got.phantoms == want.phantoms
    if labels:
        np.testing.assert_array_equal(lat.labels(), want.labels.astype(np.int32))


def _run_pair(csp, inst, ctas=0, M=None, phantoms=True, **kw):
    M = inst.M if M is None else M
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, M, trace=True, ctas=ctas, phantoms=phantoms, engine="event", **kw)
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


def test_tiny_without_phantom_count(csp):
    for seed in range(20):
        inst = synth.random_small_instance(seed, max_vertices=30, dims=(2, 3))
        _run_pair(csp, inst, ctas=1 + seed % 3, phantoms=False)


MEDIUM = [
    ([100, 80], 1, 12, 0, 120, np.uint8),
    ([100, 80], 1, 12, 0, 400, np.uint8),
    ([24, 24, 24], 1, 16, 0, 160, np.uint8),
    ([24, 24, 24], 1, 16, 1, 90, np.uint8),
    ([9, 9, 9, 9], 1, 20, 0, 200, np.uint8),
    ([300, 7], 1, 300, 0, 5000, np.uint16),
    ([2000], 1, 40, 0, 100000, np.uint16),
    ([60, 50], 1, 511, 0, 20000, np.uint16),  # max f1 = 511: the widest calendar (W = 512)
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
    got, _ = _run_pair(csp, synth.workload_64x64(), M=M)
    if M == 200:
        assert got.F1 == -1


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
    got = lat.solve(inst.A, inst.B, M, trace=True, trace_cap=4096, engine="event")
    assert list(got.answer()) == want["result"]
    assert (got.cycles, got.updates, got.launched) == (want["cycles"], want["updates"], want["launched"])
    np.testing.assert_array_equal(got.trace, np.array(want["trace"], dtype=np.int64))
    assert _digest(lat.labels()) == want["labels_sha256"]
    fast = lat.solve(inst.A, inst.B, M, engine="event")  # untraced: same answer and counts
    assert fast.answer() == got.answer()
    assert (fast.cycles, fast.updates, fast.launched) == (got.cycles, got.updates, got.launched)
    assert _digest(lat.labels()) == want["labels_sha256"]


@pytest.mark.parametrize("ctas", [1, 37, 304])
def test_cube128_independent_of_grid_size(csp, cube, ctas):
    inst, lat, g = cube
    want = g["cube3d_128_M800"]
    got = lat.solve(inst.A, inst.B, 800, ctas=ctas, engine="event")
    assert list(got.answer()) == want["result"]
    assert (got.cycles, got.updates) == (want["cycles"], want["updates"])


def test_event_equals_sweep_with_phantoms_at_size(csp):
    inst = synth.workload_cube(64, 700)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    a = lat.solve(inst.A, inst.B, 700, trace=True, phantoms=True, engine="sweep")
    la = lat.labels()
    b = lat.solve(inst.A, inst.B, 700, trace=True, phantoms=True, engine="event")
    assert a.answer() == b.answer() and (a.cycles, a.updates, a.launched, a.phantoms, a.arrivals, a.improved) == \
        (b.cycles, b.updates, b.launched, b.phantoms, b.arrivals, b.improved)
    np.testing.assert_array_equal(a.trace, b.trace)
    np.testing.assert_array_equal(la, lat.labels())
    assert b.passes == b.cycles and b.phantoms > 0
    lat.close()


@pytest.mark.parametrize("ext", [[1024, 1024], [96, 96, 96]])
def test_f2_zero_first_passage_at_size(csp, ext):
    f1, _ = synth.uniform_weights(ext, 1, 9, 21)
    f2 = np.zeros_like(f1)
    V = synth.num_vertices(ext)
    A = np.unique(synth.uniform_int(21, 3, 4, 0, V - 1))
    B = np.setdiff1d(synth.face(ext, 1, ext[1] - 1), A)
    F1, X, tau, rows = brute.dijkstra_trace(ext, f1, A, B)
    lat = csp.Lattice(ext, f1, f2)
    M = 2**31 - 2
    got = lat.solve(A, B, M, trace=True, trace_cap=1 << 15, engine="event")
    assert (got.F1, got.X, got.F2) == (F1, X, 0)
    np.testing.assert_array_equal(got.trace, rows)
    lab = lat.labels()
    reached = np.isfinite(tau) & (tau <= F1)
    assert (lab[reached] == M).all() and (lab[~reached] == 0).all()
    lat.close()


def test_edge_cases(csp):
    ext = [6, 5]
    f1, f2 = synth.uniform_weights(ext, 1, 5, 3)
    lat = csp.Lattice(ext, f1, f2)
    r = lat.solve([0], [29], 0, trace=True, engine="event")
    assert r.F1 == -1 and r.cycles == 0 and r.trace.tolist() == [[0, 0, 0]]
    a = lat.solve([0, 0, 1, 1], [29, 29], 40, trace=True, engine="event")
    b = lat.solve([1, 0], [29], 40, trace=True, engine="event")
    assert a.answer() == b.answer() and (a.trace == b.trace).all()
    for A, B, M in (([0, 1], [1], 10), ([0], [30], 10), ([], [3], 10), ([0], [3], 2**31)):
        with pytest.raises(csp.CspError) as e:
            lat.solve(A, B, M, engine="event")
        assert e.value.status == csp.ERR_INVALID
    g1, g2 = f1.copy(), f2.copy()
    g1[0, 0] = g1[1, 0] = 0
    iso = csp.Lattice(ext, g1, g2)
    r = iso.solve([0], [29], 100, trace=True, engine="event")
    assert r.F1 == -1 and r.trace.tolist() == [[0, 0, 0]]
    r = lat.solve([0], [1], 100, engine="event")
    assert r.F1 == int(f1[0, 0]) and r.cycles == 1
    lat.close()
    iso.close()


def test_engine_flags_are_exclusive(csp):
    ext = [6, 5]
    f1, f2 = synth.uniform_weights(ext, 1, 5, 3)
    lat = csp.Lattice(ext, f1, f2)
    import ctypes
    opt = csp.options()
    opt.flags = csp.OPT_EVENT | csp.OPT_SWEEP
    A = np.array([0], np.int64)
    B = np.array([29], np.int64)
    res = csp.CspResult()
    st = csp.lib().csp_solve(lat.handle, A.ctypes.data_as(csp.i64p), 1, B.ctypes.data_as(csp.i64p), 1, 40,
                             ctypes.byref(opt), ctypes.byref(res), None, 0, None)
    assert st == csp.ERR_INVALID
    lat.close()


def test_travel_times_beyond_the_window(csp):
    # f1 up to 600 (> 511): the event form refuses, the default form still solves (by the sweep)
    ext = [40, 30]
    f1, f2 = synth.uniform_weights(ext, 1, 600, 77, dtype=np.uint16)
    inst = synth.Instance(ext, f1, f2, synth.face(ext, 0, 0), synth.face(ext, 0, 39), 30000)
    lat = csp.Lattice(ext, f1, f2)
    with pytest.raises(csp.CspError) as e:
        lat.solve(inst.A, inst.B, inst.M, engine="event")
    assert e.value.status == csp.ERR_INVALID
    assert lat.default_engine() == "sweep"
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    assert lat.solve(inst.A, inst.B, inst.M).answer() == want.answer()
    lat.close()


def test_pool_growth_and_cycle_limit(csp):
    inst = synth.workload_cube(24, 300)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 300)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, 300, pool_capacity=100, trace=True, engine="event")  # doubles until it fits
    assert got.answer() == want.answer() and (got.trace == want.trace).all()
    K = 5
    cut = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 300, max_cycles=K, allow_timeout=True)
    r = lat.solve(inst.A, inst.B, 300, max_cycles=K, check=False, trace=True, engine="event")
    assert r.status == csp.ERR_TIMEOUT and r.cycles == K
    assert (r.updates, r.launched) == (cut.updates, cut.launched)
    np.testing.assert_array_equal(r.trace[:K], cut.trace[:K])
    lat.close()


def test_weights_uploaded_again(csp):
    # the edge queues are rebuilt from the new weights
    inst = synth.workload_cube(20, 260)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    lat.solve(inst.A, inst.B, 260, engine="event")
    g1, g2 = synth.uniform_weights(inst.extents, 1, 16, 99)
    lat.upload_weights(g1, g2)
    want = oracle.cycle(inst.extents, g1, g2, inst.A, inst.B, 260, labels=True)
    got = lat.solve(inst.A, inst.B, 260, trace=True, engine="event")
    _check_same(lat, got, want)
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
    for _ in range(3):  # the queues and calendar are reused
        lat.solve_async(A, B, 500, rec, trace_dev=tr, trace_cap=4096, stream=s, engine="event")
        s.synchronize()
        r = csp.result_from_record(rec.cpu().numpy())
        assert r.status == csp.OK and r.answer() == want.answer()
        n = int(rec[11].item())
        np.testing.assert_array_equal(tr[: 3 * n].view(-1, 3).cpu().numpy(), want.trace)
    t = lat.event_phase_times()
    assert t[1] > 0 and t[2] > 0
    lat.close()


# ---------------------------------------------------------------- general graphs


def _pair_graph(csp, nbr, f1, f2, A, B, M, ctas=0, directed=False):
    want = oracle.cycle_graph(nbr, f1, f2, A, B, M, labels=True)  # (one-way slots for a digraph)
    g = csp.Graph(nbr, f1, f2, directed=directed)
    got = g.solve(A, B, M, trace=True, ctas=ctas, phantoms=True, trace_cap=1 << 17, engine="event")
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched) == (want.cycles, want.updates, want.launched)
    np.testing.assert_array_equal(got.trace, want.trace)
    assert got.phantoms == want.phantoms
    np.testing.assert_array_equal(g.labels(), want.labels.astype(np.int32))
    g.close()
    return got


@pytest.mark.parametrize("seed", range(0, 120, 3))
def test_tiny_graphs(csp, seed):
    t = synth.random_small_graph(seed)
    _pair_graph(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M, ctas=1 + seed % 5)


def test_phantom_rich_tiny_graphs(csp):
    seen = 0
    for seed in range(120):
        t = synth.random_small_graph(seed, max_vertices=20, rounds=(3, 4), f_hi=20, M_max=150, max_sources=2,
                                     drop=0.2)
        seen += _pair_graph(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M).phantoms > 0
    assert seen >= 5


@pytest.mark.parametrize("side,M", [(64, 300), (256, 900)])
def test_king_graph(csp, side, M):
    g = synth.king_graph(side, 1, 16, seed=side)
    assert _pair_graph(csp, g.nbr, g.f1, g.f2, g.A, g.B, M).F1 > 0


def test_medium_random_graph(csp):
    nbr, f1, f2 = synth.random_graph(150_000, 6, seed=21, lo=1, hi=16, drop=0.1)
    A = np.arange(0, 150_000, 30_011)
    tau = brute.graph_tau(nbr, f1, A)
    B = np.argsort(-np.where(np.isfinite(tau), tau, -1), kind="stable")[:4]
    got = _pair_graph(csp, nbr, f1, f2, A, B, 120)
    assert got.F1 > 0 and got.phantoms > 0


@pytest.mark.parametrize("seed", range(0, 60, 2))
def test_tiny_digraphs(csp, seed):
    t = synth.random_small_digraph(seed)
    _pair_graph(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M, ctas=1 + seed % 5, directed=True)


def test_medium_digraph(csp):
    nbr, f1, f2 = synth.random_digraph(120_000, 6, seed=41, lo=1, hi=16, drop=0.1)
    A = np.arange(0, 120_000, 24_007)
    tau = brute.graph_tau(nbr, f1, A)
    B = np.argsort(-np.where(np.isfinite(tau), tau, -1), kind="stable")[:4]
    assert _pair_graph(csp, nbr, f1, f2, A, B, 120, directed=True).F1 > 0


# ---------------------------------------------------------------- reconstruction


@pytest.mark.parametrize("ext,M", [([64, 64], 300), ([20, 20, 20], 260)])
def test_fast_reconstruction_equals_repeated_application(csp, ext, M):
    inst = synth.workload_64x64() if ext == [64, 64] else synth.workload_cube(ext[0], M)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    path, r = lat.reconstruct_fast(inst.A, inst.B, M, engine="event")
    assert path.tolist() == want
    lat.close()


@pytest.mark.parametrize("seed", range(0, 30))
def test_fast_reconstruction_tiny(csp, seed):
    inst = synth.random_small_instance(seed, max_vertices=20)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    path, _ = lat.reconstruct_fast(inst.A, inst.B, inst.M, engine="event")
    assert (path is None and want is None) or path.tolist() == want
    lat.close()


def test_default_engine_follows_mean_travel_time(csp):
    # long travel times (mean f1 >= 64 over directed edges): the event form by default; the
    # 1-16 cube and travel times 1-64 (mean 32.5): the sweep.  Either way the solve equals the
    # oracle.
    ext = [90, 70]
    f1, f2 = synth.uniform_weights(ext, 1, 255, 91, dtype=np.uint16)
    f2 = (f2 % 16 + 1).astype(np.uint16)
    f2[f1 == 0] = 0
    inst = synth.Instance(ext, f1, f2, synth.face(ext, 0, 0), synth.face(ext, 0, 89), 1500)
    lat = csp.Lattice(ext, f1, f2)
    assert lat.default_engine() == "event"
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True, phantoms=True)
    _check_same(lat, got, want)
    lat.close()
    cube = synth.workload_cube(20, 260)
    lat = csp.Lattice(cube.extents, cube.f1, cube.f2)
    assert lat.default_engine() == "sweep"
    lat.close()
    f1, f2 = synth.uniform_weights(ext, 1, 64, 92)
    lat = csp.Lattice(ext, f1, f2)
    assert lat.default_engine() == "sweep"
    lat.close()

"""Every device-side wait of the solver is bounded, and running into a limit returns an
error status with the GPU left usable (no fault, no trap, no hang):

* the solve's watchdog (csp_options.time_limit_s) stops a long solve with CSP_ERR_TIMEOUT,
  and the rows and counts it returns are those of the cycles it completed;
* a grid barrier that one CTA never reaches (the CSP_OPT_TEST_ABSENT_CTA hook: the last
  CTA leaves before its first barrier) gives up after csp_options.barrier_us with
  CSP_ERR_BARRIER;
* a server whose session runs out while idle ends its persistent kernel, and the server is
  destroyed cleanly;
* a full query ring refuses a submission with CSP_ERR_CAPACITY;
* a reservation beyond the free device memory fails with CSP_ERR_OOM.

After each, a normal solve on the same device gives the oracle's answer.
"""
import json
import os
import time

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
def small(csp):
    inst = synth.workload_cube(24, 300)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 300)
    return inst, want


def _usable(csp, small):
    inst, want = small
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    assert lat.solve(inst.A, inst.B, 300).answer() == want.answer()
    lat.close()


@pytest.fixture(scope="module")
def slow(csp):
    # the 2048^2 anti-correlated lattice: several seconds per solve in either form
    g = json.load(open(GOLDEN))["sides"]["2048"]
    inst = synth.workload_anticorrelated(2048, M=g["M"])
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    lat.reserve(1 << 27)
    yield inst, lat
    lat.close()


@pytest.mark.parametrize("engine", ["sweep", "event"])
def test_time_limit_stops_with_completed_rows(csp, slow, small, engine):
    inst, lat = slow
    t0 = time.perf_counter()
    r = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=1 << 16, time_limit_s=1, engine=engine,
                  check=False)
    assert time.perf_counter() - t0 < 30
    assert r.status == csp.ERR_TIMEOUT
    k = r.cycles
    assert k > 100 and r.trace_len == k and r.trace.shape == (k, 3)
    # updates = the flows alive at the start of each completed cycle = live flows of rows 0 .. k-1
    assert r.updates == int(r.trace[:, 2].sum())
    # the completed rows are those of the same solve stopped by a cycle limit instead
    ref = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=1 << 16, max_cycles=k, engine=engine, check=False)
    assert ref.status == csp.ERR_TIMEOUT and ref.cycles == k
    np.testing.assert_array_equal(r.trace, ref.trace)
    assert (r.updates, r.launched) == (ref.updates, ref.launched)
    # and their beginning is the oracle's
    head = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, max_cycles=100, allow_timeout=True)
    np.testing.assert_array_equal(r.trace[:100], head.trace[:100])
    _usable(csp, small)


@pytest.mark.parametrize("engine", ["sweep", "event"])
def test_barrier_wait_gives_up(csp, small, engine):
    inst, want = small
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    t0 = time.perf_counter()
    r = lat.solve(inst.A, inst.B, 300, ctas=8, barrier_us=200_000, test_absent_cta=True, engine=engine,
                  check=False)
    assert r.status == csp.ERR_BARRIER
    assert time.perf_counter() - t0 < 10
    assert lat.solve(inst.A, inst.B, 300, ctas=8, engine=engine).answer() == want.answer()
    lat.close()
    _usable(csp, small)


def test_idle_server_session_runs_out(csp, small):
    inst, want = small
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    srv = csp.Server(lat, group_ctas=4, max_groups=2, session_seconds=1.0)
    B = inst.B[:40]  # (a server query carries at most 64 explicit targets)
    ref = lat.solve(inst.A[:64], B, 300)
    t = srv.submit(type("Q", (), {"A": inst.A[:64], "B": B, "M": 300, "axis": -1, "coord": 0})(),
                   use_hyperplane=False)
    t0 = time.perf_counter()
    r = None
    while r is None and time.perf_counter() - t0 < 10:
        r = srv.poll(t)
    assert r is not None and r.status == csp.OK and r.answer() == ref.answer()
    time.sleep(2.0)  # idle past the session: the persistent kernel gives up waiting and ends
    t0 = time.perf_counter()
    srv.close()
    assert time.perf_counter() - t0 < 5
    lat.close()
    _usable(csp, small)


def test_full_query_ring_refuses(csp, small):
    inst, want = small
    ext = [512, 512]
    f1, f2 = synth.uniform_weights(ext, 1, 16, 5)
    lat = csp.Lattice(ext, f1, f2)
    srv = csp.Server(lat, group_ctas=1, max_groups=1, queue_capacity=2, session_seconds=60.0,
                     pool_capacity=1 << 22)
    Q = type("Q", (), {})
    long_q = Q()
    long_q.A, long_q.B, long_q.M, long_q.axis, long_q.coord = synth.face(ext, 0, 0)[:64], None, 6000, 0, 511
    tickets = [srv.submit(long_q), srv.submit(long_q)]  # one CTA: these take a while each
    with pytest.raises(csp.CspError) as e:
        srv.submit(long_q)
    assert e.value.status == csp.ERR_CAPACITY
    done = {}
    t0 = time.perf_counter()
    while len(done) < 2 and time.perf_counter() - t0 < 120:
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
    assert len(done) == 2 and all(r.status == csp.OK for r in done.values())
    srv.submit(long_q)  # entries are free again
    srv.close()
    lat.close()
    _usable(csp, small)


def test_reservation_beyond_free_memory_fails(csp, small):
    torch = pytest.importorskip("torch")
    inst, want = small
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(int(free) - (2 << 30), dtype=torch.uint8, device="cuda")  # leave 2 GiB
    try:
        lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
        with pytest.raises(csp.CspError) as e:
            lat.reserve(1 << 30)  # 1 Gi flow slots: ~28 GB of pools and arrival lists
        assert e.value.status == csp.ERR_OOM
        lat.close()
    finally:
        del hog
        torch.cuda.empty_cache()
    _usable(csp, small)

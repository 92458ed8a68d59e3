"""GPU parity on general graphs (csp_create_graph): the CUDA path against the oracle's
graph form, element by element (answer, cycles, updates, flows started, trace, phantoms,
labels), on tiny random graphs (one CTA and several), phantom-rich tiny graphs, king's
graphs with 8- and 16-bit weights, a medium random graph spanning many pool tiles, a
lattice written as a graph (equal to the lattice path too), first passage at size, path
reconstruction, graphs in a batched launch next to lattices and graph queries served while
others are in flight (both equal to single solves).  All results are integers: the tolerance
is zero.
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csp():
    from paper_1511_06441_gb300 import build, csp as mod
    build.build()
    return mod


def _pair(csp, nbr, f1, f2, A, B, M, ctas=0, labels=True):
    want = oracle.cycle_graph(nbr, f1, f2, A, B, M, labels=labels)
    g = csp.Graph(nbr, f1, f2)
    got = g.solve(A, B, M, trace=True, ctas=ctas, phantoms=True, trace_cap=1 << 17)
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched) == (want.cycles, want.updates, want.launched)
    np.testing.assert_array_equal(got.trace, want.trace)
    assert got.phantoms == want.phantoms
    if labels:
        np.testing.assert_array_equal(g.labels(), want.labels.astype(np.int32))
    g.close()
    return got


@pytest.mark.parametrize("seed", range(120))
def test_tiny_graph_one_cta(csp, seed):
    t = synth.random_small_graph(seed)
    _pair(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M, ctas=1)


@pytest.mark.parametrize("seed", range(0, 120, 4))
def test_tiny_graph_many_ctas(csp, seed):
    t = synth.random_small_graph(seed)
    _pair(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M, ctas=7)


def test_phantom_rich_tiny_graphs(csp):
    seen = 0
    for seed in range(200):
        t = synth.random_small_graph(seed, max_vertices=20, rounds=(3, 4), f_hi=20, M_max=150, max_sources=2,
                                     drop=0.2)
        seen += _pair(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M).phantoms > 0
    assert seen >= 5


@pytest.mark.parametrize("side,M,wide", [(64, 300, False), (256, 900, False), (128, 200000, True)])
def test_king_graph(csp, side, M, wide):
    g = synth.king_graph(side, 1, 16, seed=side)
    f1, f2 = g.f1, g.f2
    if wide:  # 16-bit weights: f2 spread over [1, 4000]
        f1 = f1.astype(np.uint16)
        f2 = (f2.astype(np.uint16) * 250)
        f2[g.nbr < 0] = 0
    got = _pair(csp, g.nbr, f1, f2, g.A, g.B, M)
    assert got.F1 > 0


def test_medium_random_graph_spans_many_tiles(csp):
    nbr, f1, f2 = synth.random_graph(150_000, 6, seed=21, lo=1, hi=16, drop=0.1)
    A = np.arange(0, 150_000, 30_011)
    tau = brute.graph_tau(nbr, f1, A)
    B = np.argsort(-np.where(np.isfinite(tau), tau, -1), kind="stable")[:4]  # the last vertices water reaches
    got = _pair(csp, nbr, f1, f2, A, B, 120)
    assert got.F1 > 0 and int(got.trace[:, 2].max()) > 20 * 2048 and got.phantoms > 0


@pytest.mark.parametrize("which", ["64x64", "cube20"])
def test_lattice_as_graph_equals_lattice_path(csp, which):
    if which == "64x64":
        inst = synth.workload_64x64()
        Ms = (200, 400, 1000)
    else:
        ext = [20, 20, 20]
        f1, f2 = synth.uniform_weights(ext, 1, 16, 9)
        inst = synth.Instance(ext, f1, f2, synth.face(ext, 0, 0), synth.face(ext, 0, 19), 0)
        Ms = (150, 400)
    nbr, g1, g2 = synth.graph_from_lattice(inst.extents, inst.f1, inst.f2)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    gr = csp.Graph(nbr, g1, g2)
    for M in Ms:
        a = lat.solve(inst.A, inst.B, M, trace=True, phantoms=True)
        b = gr.solve(inst.A, inst.B, M, trace=True, phantoms=True)
        assert a.answer() == b.answer() and (a.cycles, a.updates, a.launched, a.phantoms) == \
            (b.cycles, b.updates, b.launched, b.phantoms)
        np.testing.assert_array_equal(a.trace, b.trace)
        np.testing.assert_array_equal(lat.labels(), gr.labels())
    lat.close()
    gr.close()


def test_first_passage_on_a_king_graph(csp):
    g = synth.king_graph(256, 1, 9, seed=5)
    f2 = np.zeros_like(g.f2)
    F1, X, tau, rows = brute.graph_dijkstra_trace(g.nbr, g.f1, g.A, g.B)
    gr = csp.Graph(g.nbr, g.f1, f2)
    got = gr.solve(g.A, g.B, 2**31 - 2, trace=True, trace_cap=1 << 15)
    assert (got.F1, got.X, got.F2) == (F1, X, 0)
    np.testing.assert_array_equal(got.trace, rows)
    gr.close()


@pytest.mark.parametrize("seed", range(0, 40))
def test_graph_reconstruction_equals_oracle(csp, seed):
    t = synth.random_small_graph(seed, max_vertices=16, rounds=(2, 4))
    want_r = oracle.cycle_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, trace=False)
    want, _ = oracle.reconstruct_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, first=want_r)
    g = csp.Graph(t.nbr, t.f1, t.f2)
    got = g.reconstruct(t.A, t.B, t.M)
    fast, r = g.reconstruct_fast(t.A, t.B, t.M)
    g.close()
    if want is None:
        assert got is None and fast is None and r.F1 == -1
    else:
        assert list(got) == want and list(fast) == want


def test_king_graph_fast_path_equals_repeated_application(csp):
    g = synth.king_graph(48, 1, 16, seed=3)
    gr = csp.Graph(g.nbr, g.f1, g.f2)
    slow = gr.reconstruct(g.A, g.B, 400)
    fast, r = gr.reconstruct_fast(g.A, g.B, 400)
    gr.close()
    assert r.F1 > 0 and list(fast) == list(slow)
    want, _ = oracle.reconstruct_graph(g.nbr, g.f1, g.f2, g.A, g.B, 400)
    assert list(fast) == want


def test_weights_of_a_graph_are_fixed(csp):
    t = synth.random_small_graph(3)
    g = csp.Graph(t.nbr, t.f1, t.f2)
    assert csp.lib().csp_upload_weights(g.handle, t.f1.ctypes.data, t.f2.ctypes.data, 0, None) == csp.ERR_INVALID
    g.close()


def test_graph_edge_cases(csp):
    # a path graph 0 - 1 - ... - 9 with one slot per direction: F1, F2 in closed form
    V = 10
    nbr = np.full((V, 2), -1, np.int64)
    nbr[:-1, 0] = np.arange(1, V)
    nbr[1:, 1] = np.arange(V - 1)
    f1 = np.where(nbr >= 0, 3, 0).astype(np.uint8)
    f2 = np.where(nbr >= 0, 2, 0).astype(np.uint8)
    g = csp.Graph(nbr, f1, f2)
    r = g.solve([0], [V - 1], 2 * (V - 1) + 1, trace=True)
    assert (r.F1, r.X, r.x_src, r.x_dir, r.F2) == (3 * (V - 1), V - 1, V - 2, 0, 2 * (V - 1))
    assert g.solve([0], [V - 1], 2 * (V - 1)).F1 == -1            # the bound is strict
    r = g.solve([0], [V - 1], 0, trace=True)                        # M <= 0: infeasible at once
    assert r.F1 == -1 and r.cycles == 0 and r.trace.tolist() == [[0, 0, 0]]
    with pytest.raises(csp.CspError):
        g.solve([0], [0], 100)                                      # A and B must be disjoint
    with pytest.raises(csp.CspError):
        g.solve([0], [V], 100)                                      # ids out of range
    g.close()
    # no edges at all: nothing flows
    e = csp.Graph(np.full((4, 3), -1, np.int64), np.zeros((4, 3), np.uint8), np.zeros((4, 3), np.uint8))
    r = e.solve([0], [3], 50, trace=True)
    assert r.F1 == -1 and r.cycles == 0
    e.close()


def test_graph_async_solve_equals_sync(csp):
    import torch
    g = synth.king_graph(96, 1, 16, seed=9)
    gr = csp.Graph(g.nbr, g.f1, g.f2)
    want = gr.solve(g.A, g.B, 500)
    gr.reserve()
    rec = torch.zeros(16, dtype=torch.int64, device="cuda")
    gr.solve_async(torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(), 500, rec)
    torch.cuda.synchronize()
    got = csp.result_from_record(rec.cpu().numpy())
    gr.close()
    assert got.status == 0 and got.answer() == want.answer() and got.updates == want.updates


def _key(r):
    return (r.answer(), r.cycles, r.updates, r.launched)


def test_batched_graphs_equal_single_solves(csp):
    # king's graphs, random graphs and lattices (same weight width) in one batched launch
    items, handles = [], []
    for i in range(18):
        if i % 3 == 0:
            side = 24 + 6 * i
            g = synth.king_graph(side, 1, 16, seed=100 + i)
            h, A, B, M = csp.Graph(g.nbr, g.f1, g.f2), g.A, g.B, 12 * side
        elif i % 3 == 1:
            V = 3000 + 700 * i
            nbr, f1, f2 = synth.random_graph(V, 6, seed=200 + i, lo=1, hi=16, drop=0.1)
            h, A, B, M = csp.Graph(nbr, f1, f2), np.array([0, V // 2]), np.arange(V - 40, V), 70
        else:
            inst = synth.workload_64x64(300 + i)
            h, A, B, M = csp.Lattice(inst.extents, inst.f1, inst.f2), inst.A, inst.B, 300
        handles.append(h)
        items.append((h, A, B, M))
    b = csp.Batch(items)
    b.run()
    got = b.results()
    single = [h.solve(A, B, M) for h, A, B, M in items]
    assert all(r.status == csp.OK for r in got)
    assert [_key(r) for r in got] == [_key(r) for r in single]
    assert sum(r.F1 > 0 for r in single) >= 12
    b.close()
    for h in handles:
        h.close()


def test_served_graph_queries_equal_alone(csp):
    nbr, f1, f2 = synth.random_graph(20_000, 6, seed=31, lo=1, hi=16, drop=0.1)
    g = csp.Graph(nbr, f1, f2)
    qs = []
    for i in range(40):
        r = synth.uniform_int(31, 1000 + i, 4, 0, 19_999)
        A = np.unique(r[:2])
        B = np.setdiff1d(synth.uniform_int(31, 2000 + i, 32, 0, 19_999), A)
        qs.append(synth.Query(A, B, 40 + 5 * (i % 9)))
    alone = [g.solve(q.A, q.B, q.M) for q in qs]
    assert max(r.max_pool for r in alone) < 1 << 16
    srv = csp.Server(g, group_ctas=4, max_groups=4, queue_capacity=16, session_seconds=120)
    got, lat_s, _ = srv.replay(qs, np.zeros(len(qs)))
    assert all(r.status == csp.OK for r in got)
    assert [_key(r) for r in got] == [_key(r) for r in alone]
    with pytest.raises(csp.CspError):   # a graph has no hyperplanes
        srv.submit(synth.Query(qs[0].A, qs[0].B, 50, 0, 0))
    srv.close()
    g.close()


# ---------------------------------------------------------------- directed graphs

def _pair_directed(csp, t_nbr, f1, f2, A, B, M, ctas=0):
    want = oracle.cycle_graph(t_nbr, f1, f2, A, B, M, labels=True)
    g = csp.Graph(t_nbr, f1, f2, directed=True)
    got = g.solve(A, B, M, trace=True, ctas=ctas, phantoms=True, trace_cap=1 << 17)
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched, got.phantoms) == \
        (want.cycles, want.updates, want.launched, want.phantoms)
    np.testing.assert_array_equal(got.trace, want.trace)
    np.testing.assert_array_equal(g.labels(), want.labels.astype(np.int32))
    g.close()
    return got


@pytest.mark.parametrize("seed", range(80))
def test_tiny_digraph(csp, seed):
    t = synth.random_small_digraph(seed)
    _pair_directed(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M, ctas=1 + seed % 5)


def test_phantom_rich_tiny_digraphs(csp):
    seen = 0
    for seed in range(150):
        t = synth.random_small_digraph(seed, max_vertices=16, rounds=(3, 5), f_hi=20, M_max=150, max_sources=2,
                                       drop=0.2)
        seen += _pair_directed(csp, t.nbr, t.f1, t.f2, t.A, t.B, t.M).phantoms > 0
    assert seen >= 3


def test_medium_digraph(csp):
    nbr, f1, f2 = synth.random_digraph(120_000, 6, seed=41, lo=1, hi=16, drop=0.1)
    A = np.arange(0, 120_000, 24_007)
    tau = brute.graph_tau(nbr, f1, A)
    B = np.argsort(-np.where(np.isfinite(tau), tau, -1), kind="stable")[:4]
    got = _pair_directed(csp, nbr, f1, f2, A, B, 120)
    assert got.F1 > 0 and int(got.trace[:, 2].max()) > 20 * 2048


def test_undirected_graph_as_digraph_is_the_same_solve(csp):
    g = synth.king_graph(96, 1, 16, seed=12)
    a = csp.Graph(g.nbr, g.f1, g.f2)
    b = csp.Graph(g.nbr, g.f1, g.f2, directed=True)   # every edge listed at both ends = two arcs
    ra = a.solve(g.A, g.B, 600, trace=True, phantoms=True)
    rb = b.solve(g.A, g.B, 600, trace=True, phantoms=True)
    assert _key(ra) == _key(rb) and ra.phantoms == rb.phantoms
    np.testing.assert_array_equal(ra.trace, rb.trace)
    a.close()
    b.close()


@pytest.mark.parametrize("seed", range(0, 30))
def test_digraph_reconstruction_equals_oracle(csp, seed):
    t = synth.random_small_digraph(seed, max_vertices=16, rounds=(2, 4))
    want_r = oracle.cycle_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, trace=False)
    want, _ = oracle.reconstruct_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, first=want_r)
    g = csp.Graph(t.nbr, t.f1, t.f2, directed=True)
    got = g.reconstruct(t.A, t.B, t.M)
    fast, r = g.reconstruct_fast(t.A, t.B, t.M)
    g.close()
    if want is None:
        assert got is None and fast is None and r.F1 == -1
    else:
        assert list(got) == want and list(fast) == want


def test_batched_digraphs_equal_single_solves(csp):
    items, handles = [], []
    for i in range(9):
        V = 2000 + 900 * i
        nbr, f1, f2 = synth.random_digraph(V, 6, seed=500 + i, lo=1, hi=16, drop=0.1)
        h = csp.Graph(nbr, f1, f2, directed=True)
        handles.append(h)
        items.append((h, np.array([0, V // 3]), np.arange(V - 30, V), 80))
    b = csp.Batch(items)
    b.run()
    got = b.results()
    single = [h.solve(A, B, M) for h, A, B, M in items]
    assert all(r.status == csp.OK for r in got)
    assert [_key(r) for r in got] == [_key(r) for r in single]
    b.close()
    for h in handles:
        h.close()


def test_served_digraph_queries_equal_alone(csp):
    nbr, f1, f2 = synth.random_digraph(20_000, 6, seed=33, lo=1, hi=16, drop=0.1)
    g = csp.Graph(nbr, f1, f2, directed=True)
    qs = []
    for i in range(30):
        r = synth.uniform_int(33, 1000 + i, 4, 0, 19_999)
        A = np.unique(r[:2])
        B = np.setdiff1d(synth.uniform_int(33, 2000 + i, 32, 0, 19_999), A)
        qs.append(synth.Query(A, B, 40 + 5 * (i % 9)))
    alone = [g.solve(q.A, q.B, q.M) for q in qs]
    assert max(r.max_pool for r in alone) < 1 << 16
    srv = csp.Server(g, group_ctas=4, max_groups=4, queue_capacity=16, session_seconds=120)
    got, _, _ = srv.replay(qs, np.zeros(len(qs)))
    srv.close()
    g.close()
    assert all(r.status == csp.OK for r in got)
    assert [_key(r) for r in got] == [_key(r) for r in alone]

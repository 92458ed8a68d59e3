"""Pins of the oracle on general graphs (Section 1 states the method for any graph; the
paper implements the bounded-degree lattice case).

* tiny random graphs: O1 and O2 against brute-force enumeration of all simple paths
  (F1, X, x, F2), O1's whole trace against the Pareto-frontier trace and its phantom count
  against the label histories (tests/brute.py);
* a lattice written as adjacency slots in its direction order gives exactly the lattice
  oracle's result, counts, trace and labels (the lattice path is pinned on its own);
* f2 = 0: the trace equals the first-passage formula (scipy Dijkstra) on king's graphs and
  random graphs;
* uniform weights on the king's graph: the closed form F1 = c1 (side - 1), F2 = c2 (side - 1);
* repeated application on a graph returns a simple path of optimal (F1, F2).
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth


def o1(g, **kw):
    return oracle.cycle_graph(g.nbr, g.f1, g.f2, g.A, g.B, g.M, **kw)


@pytest.mark.parametrize("seed", range(300))
def test_tiny_graph_answer_equals_brute_force(seed):
    g = synth.random_small_graph(seed)
    want = brute.brute_force(g)
    got = o1(g)
    assert got.answer() == (want[0], want[1], want[2], want[3], want[4])
    assert oracle.pareto_graph(g.nbr, g.f1, g.f2, g.A, g.B, g.M).answer() == got.answer()


@pytest.mark.parametrize("seed", range(0, 300, 3))
def test_tiny_graph_trace_and_phantoms(seed):
    g = synth.random_small_graph(seed, max_vertices=9)
    got = o1(g)
    np.testing.assert_array_equal(got.trace, brute.pareto_trace(g))
    assert got.phantoms == brute.phantoms(g)


def test_tiny_graphs_cover_feasible_and_infeasible():
    feasible = infeasible = 0
    for seed in range(300):
        r = o1(synth.random_small_graph(seed))
        feasible += r.F1 >= 0
        infeasible += r.F1 < 0
    assert feasible >= 100 and infeasible >= 20


def test_graph_phantoms_equal_brute_force():
    """Phantoms (flows started on a directed edge that still carries one) on denser tiny
    graphs with one or two sources and a loose bound, where labels improve several times."""
    with_phantoms = 0
    for seed in range(600):
        g = synth.random_small_graph(seed, max_vertices=20, rounds=(3, 4), f_hi=20, M_max=150, max_sources=2,
                                     drop=0.2)
        want = brute.phantoms(g)
        r = o1(g)
        assert r.phantoms == want, seed
        if want:
            np.testing.assert_array_equal(r.trace, brute.pareto_trace(g))
        with_phantoms += want > 0
    assert with_phantoms >= 20  # the comparison is not vacuous


@pytest.mark.parametrize("seed", range(40))
def test_lattice_as_graph_equals_lattice(seed):
    inst = synth.random_small_instance(seed, max_vertices=40, dims=(1, 2, 3, 4))
    nbr, g1, g2 = synth.graph_from_lattice(inst.extents, inst.f1, inst.f2)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    got = oracle.cycle_graph(nbr, g1, g2, inst.A, inst.B, inst.M, labels=True)
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched, got.phantoms) == \
        (want.cycles, want.updates, want.launched, want.phantoms)
    np.testing.assert_array_equal(got.trace, want.trace)
    np.testing.assert_array_equal(got.labels, want.labels)


def test_medium_lattice_as_graph_equals_lattice():
    inst = synth.workload_64x64()
    nbr, g1, g2 = synth.graph_from_lattice(inst.extents, inst.f1, inst.f2)
    for M in (200, 400, 1000):
        want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True)
        got = oracle.cycle_graph(nbr, g1, g2, inst.A, inst.B, M, labels=True)
        assert got.answer() == want.answer() and got.updates == want.updates
        np.testing.assert_array_equal(got.trace, want.trace)
        np.testing.assert_array_equal(got.labels, want.labels)


@pytest.mark.parametrize("kind", ["king", "random"])
def test_f2_zero_is_first_passage(kind):
    if kind == "king":
        g = synth.king_graph(40, 1, 9, seed=11)
        nbr, f1 = g.nbr, g.f1
        A, B = g.A, g.B
    else:
        nbr, f1, _ = synth.random_graph(3000, 5, seed=12, lo=1, hi=9, drop=0.2)
        A = np.arange(0, 3000, 997)
        B = np.arange(1500, 1520)
    f2 = np.zeros_like(f1)
    F1, X, tau, rows = brute.graph_dijkstra_trace(nbr, f1, A, B)
    got = oracle.cycle_graph(nbr, f1, f2, A, B, 2**31 - 2, labels=True)
    assert (got.F1, got.X) == (F1, X) and F1 > 0
    np.testing.assert_array_equal(got.trace, rows)


@pytest.mark.parametrize("c1,c2,M,side", [(3, 2, 100, 10), (3, 2, 19, 10), (3, 2, 18, 10), (1, 5, 1000, 30)])
def test_king_uniform_closed_form(c1, c2, M, side):
    g = synth.king_graph(side)
    g.f1[g.nbr >= 0] = c1
    g.f2[g.nbr >= 0] = c2
    g.M = M
    r = o1(g)
    if c2 * (side - 1) < M:
        # side - 1 king steps cross the board (one column per step), none fewer
        assert (r.F1, r.F2) == (c1 * (side - 1), c2 * (side - 1))
        assert r.X % side == side - 1
    else:
        assert r.F1 == -1


@pytest.mark.parametrize("seed", range(0, 60))
def test_graph_reconstruction_is_an_optimal_simple_path(seed):
    g = synth.random_small_graph(seed)
    r = o1(g, trace=False)
    path, _ = oracle.reconstruct_graph(g.nbr, g.f1, g.f2, g.A, g.B, g.M, first=r)
    if r.F1 < 0:
        assert path is None
        return
    assert path[0] in set(g.A.tolist()) and path[-1] == r.X and len(set(path)) == len(path)
    t = w = 0
    for a, b in zip(path, path[1:]):
        j = [k for k in range(g.S) if g.nbr[a, k] == b]
        assert len(j) == 1
        t += int(g.f1[a, j[0]])
        w += int(g.f2[a, j[0]])
    assert (t, w) == (r.F1, r.F2) and w < g.M


def _king():
    g = synth.king_graph(9)
    return g.nbr, g.f1, g.f2


def _lattice():
    i = synth.random_small_instance(5, max_vertices=60, dims=(3,))
    return synth.graph_from_lattice(i.extents, i.f1, i.f2)


@pytest.mark.parametrize("make", [_king, lambda: synth.random_graph(500, 8, seed=3, drop=0.1), _lattice])
def test_generated_graphs_are_undirected_and_simple(make):
    nbr, f1, f2 = make()
    V, S = nbr.shape
    assert S <= 8
    for v in range(V):
        row = [int(u) for u in nbr[v] if u >= 0]
        assert v not in row and len(set(row)) == len(row)           # no loop, no parallel edge
        for j in range(S):
            u = int(nbr[v, j])
            if u < 0:
                assert f1[v, j] == 0
                continue
            back = [k for k in range(S) if nbr[u, k] == v]
            assert len(back) == 1 and f1[v, j] >= 1
            assert (f1[u, back[0]], f2[u, back[0]]) == (f1[v, j], f2[v, j])


def test_king_graph_interior_degree_is_eight():
    g = synth.king_graph(6)
    deg = (g.nbr >= 0).sum(1).reshape(6, 6)
    assert (deg[1:-1, 1:-1] == 8).all() and deg[0, 0] == 3 and deg[0, 3] == 5


# ---------------------------------------------------------------- directed graphs

@pytest.mark.parametrize("seed", range(300))
def test_tiny_digraph_answer_equals_brute_force(seed):
    g = synth.random_small_digraph(seed)
    want = brute.brute_force(g)
    got = o1(g)
    assert got.answer() == tuple(want[:5])
    assert oracle.pareto_graph(g.nbr, g.f1, g.f2, g.A, g.B, g.M).answer() == got.answer()


def test_digraph_trace_and_phantoms_equal_brute_force():
    with_phantoms = feasible = 0
    for seed in range(400):
        g = synth.random_small_digraph(seed, max_vertices=16, rounds=(3, 5), f_hi=20, M_max=150, max_sources=2,
                                       drop=0.2)
        r = o1(g)
        np.testing.assert_array_equal(r.trace, brute.pareto_trace(g))
        assert r.phantoms == brute.phantoms(g), seed
        with_phantoms += r.phantoms > 0
        feasible += r.F1 >= 0
    assert with_phantoms >= 10 and feasible >= 100


def test_digraph_f2_zero_is_first_passage():
    nbr, f1, _ = synth.random_digraph(4000, 5, seed=13, lo=1, hi=9, drop=0.2)
    A = np.array([0, 1999])
    B = np.arange(3000, 3030)
    F1, X, tau, rows = brute.graph_dijkstra_trace(nbr, f1, A, B)
    got = oracle.cycle_graph(nbr, f1, np.zeros_like(f1), A, B, 2**31 - 2)
    assert (got.F1, got.X) == (F1, X) and F1 > 0
    np.testing.assert_array_equal(got.trace, rows)


def test_random_digraph_degrees():
    nbr, f1, f2 = synth.random_digraph(1000, 8, seed=5, drop=0.1)
    indeg = np.bincount(nbr[nbr >= 0], minlength=1000)
    assert indeg.max() <= 8 and (nbr != np.arange(1000)[:, None]).all()
    for v in range(1000):
        row = [int(u) for u in nbr[v] if u >= 0]
        assert len(set(row)) == len(row)
    assert ((nbr >= 0) == (f1 > 0)).all()


def test_slots_from_edges_round_trip():
    from paper_1511_06441_gb300 import csp
    nbr, f1, f2 = synth.random_graph(300, 5, seed=4, drop=0.2)
    V, S = nbr.shape
    E = [(v, int(nbr[v, j]), int(f1[v, j]), int(f2[v, j])) for v in range(V) for j in range(S)
         if nbr[v, j] > v]
    edges = np.array([(a, b) for a, b, _, _ in E])
    n2, g1, g2 = csp.slots_from_edges(V, edges, np.array([w for *_, w, _ in E], np.uint8),
                                      np.array([w for *_, w in E], np.uint8))
    # the same undirected graph: the same edge set with the same weights, one slot per end
    def edge_set(n, a1, a2):
        return {(v, int(n[v, j]), int(a1[v, j]), int(a2[v, j])) for v in range(n.shape[0])
                for j in range(n.shape[1]) if n[v, j] >= 0}
    assert edge_set(n2, g1, g2) == edge_set(nbr, f1, f2)
    # an oracle solve sees the same problem (slot order only renames directions)
    A, B = [0, 1], list(range(250, 260))
    a = oracle.cycle_graph(nbr, f1, f2, A, B, 60)
    b = oracle.cycle_graph(n2, g1, g2, A, B, 60)
    assert (a.F1, a.X, a.F2, a.updates) == (b.F1, b.X, b.F2, b.updates)
    np.testing.assert_array_equal(a.trace, b.trace)


def test_slots_from_edges_directed_and_limits():
    from paper_1511_06441_gb300 import csp
    nbr, f1, f2 = csp.slots_from_edges(3, [(0, 1), (0, 2), (2, 1)], np.array([1, 2, 3], np.uint8),
                                       np.array([4, 5, 6], np.uint8), directed=True)
    assert nbr.tolist() == [[1, 2], [-1, -1], [1, -1]]
    assert f1.tolist() == [[1, 2], [0, 0], [3, 0]] and f2.tolist() == [[4, 5], [0, 0], [6, 0]]
    star = [(0, k) for k in range(1, 10)]
    with pytest.raises(ValueError):
        csp.slots_from_edges(10, star, np.ones(9, np.uint8), np.ones(9, np.uint8))


@pytest.mark.parametrize("seed", range(0, 60))
def test_digraph_reconstruction_is_an_optimal_simple_path(seed):
    g = synth.random_small_digraph(seed)
    r = o1(g, trace=False)
    path, _ = oracle.reconstruct_graph(g.nbr, g.f1, g.f2, g.A, g.B, g.M, first=r)
    want = brute.brute_force(g)
    if r.F1 < 0:
        assert path is None and want[0] == -1
        return
    assert path[0] in set(g.A.tolist()) and path[-1] == r.X and len(set(path)) == len(path)
    t = w = 0
    for a, b in zip(path, path[1:]):                  # every step follows an arc a -> b
        j = [k for k in range(g.S) if g.nbr[a, k] == b]
        assert len(j) == 1
        t += int(g.f1[a, j[0]])
        w += int(g.f2[a, j[0]])
    assert (t, w) == (r.F1, r.F2) == (want[0], want[4]) and w < g.M

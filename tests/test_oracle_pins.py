"""Pins of the CPU oracle against things other than itself (no GPU).

* brute force over all simple paths (Section 1 definition) on tiny lattices: F1, F2, X, x
  for O1 and O2, and the full per-cycle trace of O1 from per-vertex Pareto frontiers;
* f2 = 0 reduces the problem to first-passage percolation (Section 2): F1 and the whole
  trace of O1 equal what plain Dijkstra (scipy) implies, at sizes brute force cannot reach;
* closed forms: uniform weights (F1 = c1 * L1 distance iff c2 * distance < M) and a path
  graph (F1, F2 are plain sums; the bound is strict);
* monotonicity of F1 in M;
* the active set on the lattice of the paper's Lemma (Section "Large sets of active
  vertices"), in tests/test_lemma_golden.py.
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth


def _tiny(seed, **kw):
    return synth.random_small_instance(seed, **kw)


@pytest.mark.parametrize("seed", range(0, 160))
def test_o1_o2_equal_brute_force_tiny(seed):
    inst = _tiny(seed)
    want = brute.brute_force(inst)
    o1 = oracle.solve_instance(inst)
    o2 = oracle.pareto(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    assert o1.answer() == want, (inst.extents, inst.A, inst.B, inst.M)
    assert o2.answer() == want


@pytest.mark.parametrize("seed", range(1000, 1080))
def test_o1_trace_equals_pareto_frontier_formula(seed):
    inst = _tiny(seed, max_vertices=12)
    got = oracle.solve_instance(inst)
    want = brute.pareto_trace(inst)
    np.testing.assert_array_equal(got.trace, want)
    assert got.cycles == len(want) - 1
    assert got.updates == int(want[:-1, 2].sum())


@pytest.mark.parametrize("seed", range(2000, 2040))
def test_o1_trace_equals_pareto_frontier_formula_larger_M(seed):
    # same check with a loose bound, so many labels improve several times (phantoms)
    inst = _tiny(seed, max_vertices=12, f_lo=(1,))
    inst.M = 40
    got = oracle.solve_instance(inst)
    np.testing.assert_array_equal(got.trace, brute.pareto_trace(inst))


def test_planted_mistakes_are_caught_by_brute_force():
    # A plausible slip (dropping the f2 term, or a non-strict bound) changes the answer
    # on some tiny instance; the brute-force pins above would see it.
    changed_f2, changed_strict = 0, 0
    for seed in range(200):
        inst = _tiny(seed)
        want = brute.brute_force(inst)
        zero = synth.Instance(inst.extents, inst.f1, np.zeros_like(inst.f2), inst.A, inst.B, inst.M)
        if oracle.solve_instance(zero).answer() != want:
            changed_f2 += 1
        loose = synth.Instance(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M + 1)
        if oracle.solve_instance(loose).answer() != want:
            changed_strict += 1
    assert changed_f2 > 10 and changed_strict > 10


@pytest.mark.parametrize("seed,ext", [(11, [40, 40]), (12, [16, 16, 16]), (13, [300]), (14, [12, 10, 9, 8])])
def test_f2_zero_is_first_passage_percolation(seed, ext):
    f1, _ = synth.uniform_weights(ext, 1, 9, seed)
    # knock out ~10% of the edges to make it a lattice subgraph
    holes = synth.uniform_unit(seed, 77, f1.size).reshape(f1.shape) < 0.1
    f1[holes] = 0
    f2 = np.zeros_like(f1)
    V = synth.num_vertices(ext)
    A = np.unique(synth.uniform_int(seed, 3, 5, 0, V - 1))
    B = np.setdiff1d(np.unique(synth.uniform_int(seed, 4, 40, 0, V - 1)), A)
    F1, X, tau, rows = brute.dijkstra_trace(ext, f1, A, B)
    got = oracle.cycle(ext, f1, f2, A, B, 2**31 - 1, labels=True)
    assert got.F1 == F1 and got.X == X
    if F1 >= 0:
        assert got.F2 == 0
        # x: the smallest (Y, dir) with tau(Y) + f1(Y, X) == F1
        adj, _ = brute.directed_edges(ext, f1, f2)
        cands = sorted((u, d ^ 1) for (u, d, t1, _) in adj[X] if tau[u] + t1 == F1)
        assert (got.x_src, got.x_dir) == cands[0]
    np.testing.assert_array_equal(got.trace, rows)


@pytest.mark.parametrize("c1,c2,M", [(3, 2, 100), (3, 2, 17), (3, 2, 16), (1, 5, 1000), (7, 0, 1)])
def test_uniform_weights_closed_form(c1, c2, M):
    ext = [9, 7]
    V = 63
    f1 = np.full((2, V), c1, np.uint8)
    f2 = np.full((2, V), c2, np.uint8)
    up = synth.upper_face_mask(ext)
    f1[up] = 0
    f2[up] = 0
    A = synth.vertex_id(np.array([[1, 1]]), ext)
    B = synth.vertex_id(np.array([[7, 5], [8, 0]]), ext)
    # every path needs at least the L1 distance in edges: 10 to (7,5), 8 to (8,0)
    dist, X = 8, int(synth.vertex_id(np.array([[8, 0]]), ext)[0])
    inst = synth.Instance(ext, f1, f2, A, B, M)
    for r in (oracle.solve_instance(inst), oracle.pareto(ext, f1, f2, A, B, M)):
        if c2 * dist < M:
            assert (r.F1, r.X, r.F2) == (c1 * dist, X, c2 * dist)
        else:
            assert r.F1 == -1


def test_path_graph_sums_and_strict_bound():
    n = 50
    f1 = synth.uniform_int(9, 1, n, 1, 9).reshape(1, n)
    f2 = synth.uniform_int(9, 2, n, 0, 9).reshape(1, n)
    f1[0, -1] = f2[0, -1] = 0
    T, W = int(f1[0, :-1].sum()), int(f2[0, :-1].sum())
    for M, ok in ((W + 1, True), (W, False), (10**6, True)):
        r = oracle.cycle([n], f1, f2, [0], [n - 1], M)
        p = oracle.pareto([n], f1, f2, [0], [n - 1], M)
        if ok:
            assert r.answer() == (T, n - 1, n - 2, 0, W) == p.answer()
            assert r.cycles == n - 1  # one cycle per edge on a path
        else:
            assert r.F1 == -1 and p.F1 == -1


def test_monotone_in_M():
    inst = synth.workload_64x64()
    prev = None
    for M in (200, 230, 231, 240, 260, 300, 363, 364, 500):
        r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, trace=False)
        F1 = r.F1 if r.F1 >= 0 else np.inf
        if prev is not None:
            assert F1 <= prev
        if r.F1 >= 0:
            assert r.F2 < M
        prev = F1


def test_o1_equals_o2_medium():
    for seed in range(5):
        ext = [24, 20] if seed % 2 else [9, 8, 7]
        f1, f2 = synth.uniform_weights(ext, 1, 12, 100 + seed)
        V = synth.num_vertices(ext)
        A = synth.face(ext, 0, 0)
        B = synth.face(ext, 0, ext[0] - 1)
        for M in (40, 80, 160):
            a = oracle.cycle(ext, f1, f2, A, B, M, trace=False)
            b = oracle.pareto(ext, f1, f2, A, B, M)
            assert a.answer() == b.answer()


def test_invalid_inputs():
    ext = [4, 4]
    f1, f2 = synth.uniform_weights(ext, 1, 3, 1)
    with pytest.raises(oracle.OracleError):
        oracle.cycle(ext, f1, f2, [0, 1], [1, 15], 10)   # A and B overlap
    with pytest.raises(oracle.OracleError):
        oracle.cycle(ext, f1, f2, [0], [16], 10)         # id out of range
    with pytest.raises(oracle.OracleError):
        oracle.pareto(ext, f1, f2, [], [3], 10)          # empty A
    # M <= 0 is not an error: no walk has F2 < M
    assert oracle.cycle(ext, f1, f2, [0], [15], 0).F1 == -1
    assert oracle.pareto(ext, f1, f2, [0], [15], -5).F1 == -1


def test_duplicates_in_A_and_B_are_sets():
    inst = synth.workload_64x64()
    a = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, 300)
    A2 = np.concatenate([inst.A, inst.A[::-1]])
    B2 = np.concatenate([inst.B, inst.B[:5]])
    b = oracle.cycle(inst.extents, inst.f1, inst.f2, A2, B2, 300)
    assert a.answer() == b.answer()
    np.testing.assert_array_equal(a.trace, b.trace)


# ---------------------------------------------------------------- unconstrained lexicographic optimum

BIG_M = (1 << 31) - 2


@pytest.mark.parametrize("seed", range(2000, 2060))
def test_lexmin_equals_brute_force_without_bound(seed):
    """With no binding bound the answer is the lexicographic (F1, F2) optimum; brute force
    over simple paths gives it with the same tie rules for X and x."""
    inst = _tiny(seed)
    inst.M = BIG_M
    F1, X, xs, xd, F2 = brute.brute_force(inst)
    assert oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, full=True) == (F1, F2, X, xs, xd)


@pytest.mark.parametrize("seed", range(2100, 2140))
def test_lexmin_is_the_answer_where_the_bound_does_not_bind(seed):
    """Section 1: if the lightest fastest walk satisfies F2 < M, the cycle loop returns it."""
    inst = _tiny(seed)
    F1, F2, X, xs, xd = oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, full=True)
    if F1 < 0:
        return
    inst.M = F2 + 1 + seed % 7
    assert oracle.solve_instance(inst).answer() == (F1, X, xs, xd, F2)


def _scipy_lexmin(inst):
    """(F1, F2, X, x_src, x_dir) from scipy's Dijkstra on the composite weight f1 * 2^25 + f2
    (exact in float64 at these sizes), x by the smallest (predecessor, direction) among the
    neighbours Y of X with dist(Y) + w(Y, X) = dist(X)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    S = float(1 << 25)
    adj, V = brute.directed_edges(inst.extents, inst.f1, inst.f2)
    rows, cols, wts = [], [], []
    for v, es in adj.items():
        for u, _, t1, w1 in es:
            rows.append(v)
            cols.append(u)
            wts.append(t1 * S + w1)
    G = csr_matrix((np.array(wts), (np.array(rows), np.array(cols))), shape=(V, V))
    dist = dijkstra(G, indices=sorted(set(int(a) for a in inst.A)), min_only=True)
    B = sorted(set(int(b) for b in inst.B))
    X = min(B, key=lambda b: (dist[b], b))
    best = None
    for u, dr, t1, w1 in adj[X]:
        if dist[u] + (t1 * S + w1) == dist[X]:
            key = (u, dr ^ 1)  # the edge leaves u towards X in the reverse direction
            best = key if best is None else min(best, key)
    F1, F2 = int(dist[X] // S), int(dist[X] % S)
    return F1, F2, X, best[0], best[1]


@pytest.mark.parametrize("side,seed", [(48, 3), (64, 11), (96, 12)])
def test_lexmin_equals_scipy_dijkstra_on_anticorrelated_lattices(side, seed):
    inst = synth.workload_anticorrelated(side, seed=seed)
    assert oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, full=True) == _scipy_lexmin(inst)


@pytest.mark.parametrize("seed", range(2200, 2260))
def test_lexmin_path_equals_repeated_application_where_the_bound_does_not_bind(seed):
    """The Dijkstra predecessor chain is a second, independent route to the path that
    repeated application of the cycle loop finds (Section 1) when the bound does not bind;
    on tiny lattices its sums are also the brute-force optimum."""
    inst = _tiny(seed)
    F1, F2, X, xs, xd, path = oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, path=True)
    if F1 < 0:
        assert path is None
        return
    inst.M = F2 + 1 + seed % 5
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    assert path == want
    assert path[-1] == X and (len(path) == 1 or path[-2] == xs)
    assert brute.brute_force(inst) == (F1, X, xs, xd, F2)


def test_lexmin_path_on_anticorrelated_lattice_matches_repeated_application():
    inst = synth.workload_anticorrelated(40, seed=7)
    F1, F2, X, xs, xd, path = oracle.lexmin(inst.extents, inst.f1, inst.f2, inst.A, inst.B, path=True)
    inst.M = (12 * F2) // 10
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    assert path == want and path[0] == 0 and path[-1] == X


# ---------------------------------------------------------------- phantoms (Step 5)

def test_o1_phantoms_equal_brute_force():
    """Flows started on an edge that already carries one, counted by O1 (per-edge counts of
    live flows) against the definition on all simple paths' label histories."""
    with_phantoms = 0
    for seed in range(4000, 4300):
        inst = _tiny(seed, max_vertices=18, dims=(2,), f_lo=(0,), f_hi=12, absent_prob=0.0)
        inst.M = 80
        want = brute.phantoms(inst)
        assert oracle.solve_instance(inst).phantoms == want, seed
        with_phantoms += want > 0
    assert with_phantoms >= 20  # the comparison is not vacuous


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_no_phantoms_when_weights_are_zero(seed):
    """With f2 = 0 every label jumps to M at its first arrival and never improves again, so no
    vertex starts a second flow on an edge."""
    inst = synth.workload_point_source(48, seed=seed)
    r = oracle.cycle(inst.extents, inst.f1, np.zeros_like(inst.f2), inst.A, inst.B, 1, trace=False)
    assert r.phantoms == 0 and r.launched > 0

"""Pins of the oracle's path reconstruction (repeated application, Section 1).

The recurrence read here is B' = {Y}, M' = F2 - f2(x) + 1, V' = V minus (B and the path
found so far), A' = A.  Checked against brute force: the returned path is a simple path
of the lattice from A to X whose travel time and weight are the optimum's (F1, F2); and
every step removes exactly the last edge: F1' = F1 - f1(x), F2' = F2 - f2(x).
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth


def _check_path(inst, path, F1, F2, X):
    adj, V = brute.directed_edges(inst.extents, inst.f1, inst.f2)
    assert path[0] in set(inst.A.tolist()) and path[-1] == X
    assert len(set(path)) == len(path)  # simple
    t = w = 0
    for a, b in zip(path, path[1:]):
        e = [(u, d, t1, w1) for (u, d, t1, w1) in adj[a] if u == b]
        assert e, (a, b)
        t += e[0][2]
        w += e[0][3]
    assert (t, w) == (F1, F2)
    assert F2 < inst.M


@pytest.mark.parametrize("seed", range(0, 120))
def test_reconstruction_is_an_optimal_path(seed):
    inst = synth.random_small_instance(seed, max_vertices=16)
    want = brute.brute_force(inst)
    path, steps = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    if want[0] < 0:
        assert path is None
        return
    F1, X, _, _, F2 = want
    _check_path(inst, path, F1, F2, X)
    for a, b in zip(steps, steps[1:]):
        t1, w1 = oracle.edge_weight(inst.extents, inst.f1, inst.f2, a.x_src, a.x_dir)
        assert (b.F1, b.F2) == (a.F1 - t1, a.F2 - w1)


def test_reconstruction_64x64():
    inst = synth.workload_64x64()
    inst.M = 300  # M = 200 is infeasible on this lattice
    path, steps = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    _check_path(inst, path, steps[0].F1, steps[0].F2, steps[0].X)
    assert len(steps) == len(path) - 1


def test_paper_literal_bound_loses_paths():
    # With the strict bound F2 < M (Section 1), the literal M' = F2 - f2(x) excludes the
    # sub-path itself (its weight is exactly F2 - f2(x)); the +1 of the reading is needed.
    lost = 0
    for seed in range(60):
        inst = synth.random_small_instance(seed, max_vertices=16)
        r = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, trace=False)
        if r.F1 < 0 or r.x_src in set(inst.A.tolist()):
            continue
        _, w2 = oracle.edge_weight(inst.extents, inst.f1, inst.f2, r.x_src, r.x_dir)
        removed = sorted(set(inst.B.tolist()))
        lit = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, [r.x_src], r.F2 - w2, trace=False,
                           removed=removed)
        good = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, [r.x_src], r.F2 - w2 + 1, trace=False,
                            removed=removed)
        assert good.F1 == r.F1 - oracle.edge_weight(inst.extents, inst.f1, inst.f2, r.x_src, r.x_dir)[0]
        lost += lit.F1 != good.F1
    assert lost > 0

"""The active set on the lattice of the paper's Lemma (Section "Large sets of active
vertices", the Lemma before Theorem 2).

Lattice V_n = [-n, n] x [0, n]; edges on the y axis have travel time 1, all others 2;
weights play no role (M = infinity, here f2 = 0 and M = 2^31 - 1); water starts on the
whole x axis.  The Lemma lists, for every time T, a set of active vertices.  Under the
paper's own definition of an active vertex (a vertex that is the source of an active
edge), the listed set is contained in the true active set, which also holds the
vertices (+-k, T - 2k - 1) beside the staircase; the true set is exactly
{v : tau(v) <= T < tau(w) for some neighbour w}, tau the first-passage time (plain
Dijkstra).  Both facts are checked here on the oracle's snapshot.
"""
import json
import os

import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lemma_active_set.json")


def lemma_lattice(n):
    ext = [2 * n + 1, n + 1]          # x' = x + n in [0, 2n], y in [0, n]
    V = synth.num_vertices(ext)
    f1 = np.full((2, V), 2, np.uint8)
    f2 = np.zeros((2, V), np.uint8)
    c = synth.coords(np.arange(V), ext)
    f1[1, c[:, 0] == n] = 1           # vertical edges on the y axis
    up = synth.upper_face_mask(ext)
    f1[up] = 0
    A = synth.face(ext, 1, 0)
    B = synth.face(ext, 1, n)
    return ext, f1, f2, A, B


def lemma_set(T, n):
    """The set printed in the Lemma, clipped to |x| <= n."""
    K = (T + 1) // 4
    pts = {(0, T), (0, T - 1)}
    for k in range(1, K + 1):
        pts |= {(-k, T - 2 * k), (k, T - 2 * k)}
    for z in range(-n, n + 1):
        if abs(z) > K:
            pts.add((z, T // 2))
    return pts


def test_golden_fixture_matches_formula():
    g = json.load(open(GOLDEN))
    n = g["n"]
    for T, listed in g["lemma_sets"].items():
        assert {tuple(p) for p in listed} == lemma_set(int(T), n)


@pytest.mark.parametrize("T", list(range(3, 23)))
def test_lemma_set_is_contained_in_the_active_set(T):
    n = 24
    ext, f1, f2, A, B = lemma_lattice(n)
    r = oracle.cycle(ext, f1, f2, A, B, 2**31 - 1, snap_time=T)
    c = synth.coords(r.snapshot, ext)
    active = {(int(x) - n, int(y)) for x, y in c}
    listed = lemma_set(T, n)
    assert listed <= active
    # the vertices the Lemma leaves out are exactly the staircase neighbours (+-k, T-2k-1)
    extra = active - listed
    assert all(y == T - 2 * abs(x) - 1 for x, y in extra)
    # and the whole set is the first-passage formula
    t = brute.tau(ext, f1, A)
    adj, V = brute.directed_edges(ext, f1, f2)
    want = {v for v in range(V) if t[v] <= T and any(t[u] > T for (u, _, _, _) in adj[v])}
    assert set(int(v) for v in r.snapshot) == want

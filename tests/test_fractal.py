"""The environments omega_j of the paper's t log t construction (proof of Theorem 3,
Section "Large sets of active vertices") and the oracle's active-set count on them.

The generator is checked against the construction written out with explicit
coordinates for omega_1, omega_2 and omega_3 and against its structure (nesting,
mirror symmetry).
With f2 = 0 the oracle's whole trace on omega_j must equal the first-passage formula
(plain Dijkstra).  The last test pins a lattice fact behind the measured trend: the
segment LO, a time-1 staircase starting on the source line, shortens no first-passage
time by more than one unit.
"""
import numpy as np
import pytest

import brute
import oracle
from paper_1511_06441_gb300 import synth


def fast_edges(inst):
    """{("h"|"v", x, y)}: the time-1 edges, (x, y) -> (x + 1, y) or (x, y) -> (x, y + 1)."""
    W, H = inst.extents
    t = (W - 1) // 2
    out = set()
    for k, tag in ((0, "h"), (1, "v")):
        for v in np.flatnonzero(inst.f1[k] == 1):
            out.add((tag, int(v % W) - t, int(v // W)))
    return out


def staircase(px, py, m):
    """The slope-1 staircase from (px, py): up, then right, m times."""
    s = set()
    for i in range(m):
        s.add(("v", px + i, py + i))
        s.add(("h", px + i, py + i + 1))
    return s


def mirror(edges):
    out = set()
    for tag, x, y in edges:
        out.add((tag, -x, y) if tag == "v" else (tag, -x - 1, y))
    return out


@pytest.mark.parametrize("t", [2, 4, 16, 64])
def test_omega1_is_the_y_axis_and_LO(t):
    inst = synth.fractal_environment(t, 1)
    assert inst.extents == [2 * t + 1, t + 2]
    want = {("v", 0, y) for y in range(t + 1)}
    lo = staircase(-t // 2, 0, t // 2)         # L = (-t/2, 0) to O = (0, t/2)
    want |= lo | mirror(lo)
    assert fast_edges(inst) == want
    # every other edge takes 2; the upper faces hold no edge; weights are 0
    W, H = inst.extents
    c = synth.coords(np.arange(inst.V), inst.extents)
    assert (inst.f1[0][c[:, 0] == W - 1] == 0).all() and (inst.f1[1][c[:, 1] == H - 1] == 0).all()
    inner = np.stack([c[:, 0] < W - 1, c[:, 1] < H - 1])
    assert set(np.unique(inst.f1[inner]).tolist()) <= {1, 2}
    assert not inst.f2.any()
    np.testing.assert_array_equal(inst.A, np.arange(W))
    np.testing.assert_array_equal(inst.B, np.arange(W) + W * (H - 1))


@pytest.mark.parametrize("t", [4, 16, 64])
def test_omega2_adds_L0X_and_XT0(t):
    # L0 = (-t/4, t/4), X = (-t/4, t/2), T0 = (0, 3t/4)
    one = fast_edges(synth.fractal_environment(t, 1))
    two = fast_edges(synth.fractal_environment(t, 2))
    seg = {("v", -t // 4, y) for y in range(t // 4, t // 2)} | staircase(-t // 4, t // 2, t // 4)
    assert two == one | seg | mirror(seg)


@pytest.mark.parametrize("t", [8, 64])
def test_omega3_halves_both_triangles(t):
    # the halves of LOT are (L, L0, X) with L = (-t/2, 0), s = t/4 and (X, T0, T) with
    # X = (-t/4, t/2), s = t/4; in each, the vertical from L + (t/8, t/8) to L + (t/8, t/4)
    # and the staircase from L + (t/8, t/4) of length t/8 become fast
    two = fast_edges(synth.fractal_environment(t, 2))
    three = fast_edges(synth.fractal_environment(t, 3))
    h = t // 8
    seg = set()
    for lx, ly in ((-t // 2, 0), (-t // 4, t // 2)):
        seg |= {("v", lx + h, y) for y in range(ly + h, ly + 2 * h)} | staircase(lx + h, ly + 2 * h, h)
    assert three == two | seg | mirror(seg)


@pytest.mark.parametrize("t", [8, 64])
def test_nested_and_mirrored(t):
    k = t.bit_length() - 1
    prev = set()
    for j in range(1, k + 1):
        e = fast_edges(synth.fractal_environment(t, j))
        assert prev < e
        assert mirror(e) == e
        prev = e


def test_rejects_bad_arguments():
    for t, j in [(1, 1), (12, 1), (16, 0), (16, 5)]:
        with pytest.raises(ValueError):
            synth.fractal_environment(t, j)


@pytest.mark.parametrize("t,j", [(8, 1), (8, 3), (16, 1), (16, 2), (16, 4), (32, 1), (32, 3), (32, 5)])
def test_oracle_trace_is_first_passage(t, j):
    inst = synth.fractal_environment(t, j)
    F1, X, tau, rows = brute.dijkstra_trace(inst.extents, inst.f1, inst.A, inst.B)
    got = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    assert (got.F1, got.X, got.F2) == (F1, X, 0) == (t + 1, X, 0)
    assert X == (inst.extents[1] - 1) * inst.extents[0] + t   # the top of the y axis
    np.testing.assert_array_equal(got.trace, rows)
    # every time 0..t+1 is a cycle (the y axis delivers one arrival per unit of time)
    np.testing.assert_array_equal(got.trace[:, 0], np.arange(t + 2))


@pytest.mark.parametrize("t", [16, 64, 256])
def test_LO_shortens_first_passage_by_at_most_one(t):
    # LO starts on the source line: its time-1 staircase gains one unit of height per two
    # units of time, as a time-2 vertical edge does, so against the Lemma's lattice (the
    # y axis alone fast) omega_1 reaches no vertex more than one unit sooner
    inst = synth.fractal_environment(t, 1)
    W, H = inst.extents
    c = synth.coords(np.arange(inst.V), inst.extents)
    lemma = np.where(inst.f1 > 0, 2, 0).astype(np.uint8)
    lemma[1, (c[:, 0] == t) & (c[:, 1] < H - 1)] = 1
    t1 = brute.tau(inst.extents, inst.f1, inst.A)
    t0 = brute.tau(inst.extents, lemma, inst.A)
    gain = t0 - t1
    assert gain.min() == 0 and gain.max() == 1
    # the staircase's lower end: (-t/2, 1) is reached at time 1 by its first (vertical) edge
    assert t1[W + t - t // 2] == 1 and t0[W + t - t // 2] == 2
    # the y axis (time 1) reaches (0, y) at time y in both
    np.testing.assert_array_equal(t1[np.arange(H) * W + t], np.arange(H))

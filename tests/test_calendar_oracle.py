"""O4, the cycle loop driven by events (per-edge flow queues, arrival-time buckets), against
O1: the same answer, cycle and work counts, phantoms, trace and labels on every instance,
which checks the reorganisation the calendar-queue design relies on (arrivals and removals
both take from the front of an edge's queue; a cycle touches only its events).  O1 is pinned
against brute force and first passage on its own (tests/test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
from paper_1511_06441_gb300 import synth


def _same(a, b):
    assert a.answer() == b.answer()
    assert (a.cycles, a.updates, a.launched, a.phantoms) == (b.cycles, b.updates, b.launched, b.phantoms)
    np.testing.assert_array_equal(a.trace, b.trace)
    if a.labels is not None:
        np.testing.assert_array_equal(a.labels, b.labels)


def _conserved(r):
    # every pushed flow either arrived, was removed, or is still in flight at the end
    ev = r.events
    assert ev["pushes"] == r.launched
    assert ev["pushes"] - ev["arrivals"] - ev["removals"] == int(r.trace[-1, 2])


@pytest.mark.parametrize("seed", range(300))
def test_tiny_lattices(seed):
    inst = synth.random_small_instance(seed, max_vertices=30, dims=(1, 2, 3, 4))
    a = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    b = oracle.calendar(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    _same(a, b)
    _conserved(b)


@pytest.mark.parametrize("seed", range(0, 300, 2))
def test_tiny_graphs_and_digraphs(seed):
    for t in (synth.random_small_graph(seed, max_vertices=20, rounds=(2, 4), f_hi=20, M_max=150),
              synth.random_small_digraph(seed, max_vertices=16, rounds=(3, 5), f_hi=20, M_max=150, max_sources=2)):
        a = oracle.cycle_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, labels=True)
        b = oracle.calendar_graph(t.nbr, t.f1, t.f2, t.A, t.B, t.M, labels=True)
        _same(a, b)
        _conserved(b)


@pytest.mark.parametrize("M", [200, 250, 400, 1000])
def test_64x64(M):
    i = synth.workload_64x64()
    a = oracle.cycle(i.extents, i.f1, i.f2, i.A, i.B, M, labels=True)
    b = oracle.calendar(i.extents, i.f1, i.f2, i.A, i.B, M, labels=True)
    _same(a, b)
    _conserved(b)


def test_medium_cube_and_wide_weights():
    ext = [24, 24, 24]
    f1, f2 = synth.uniform_weights(ext, 1, 16, 2)
    A, B = synth.face(ext, 0, 0), synth.face(ext, 0, 23)
    for M in (150, 300):
        _same(oracle.cycle(ext, f1, f2, A, B, M, labels=True), oracle.calendar(ext, f1, f2, A, B, M, labels=True))
    # 16-bit weights, travel times up to 255 (time buckets wrap after 256 units)
    inst = synth.workload_anticorrelated(96)
    M = 1200 * 96
    _same(oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True),
          oracle.calendar(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M, labels=True))


def test_first_passage_and_fractal_environment():
    inst = synth.fractal_environment(32, 4)
    a = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    b = oracle.calendar(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    _same(a, b)
    assert b.phantoms == 0 and b.events["removals"] > 0

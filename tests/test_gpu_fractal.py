"""GPU parity on the environments omega_j of the paper's t log t construction (proof of
Theorem 3): the CUDA path's trace, result and labels against the oracle at t = 32, its
whole trace against the first-passage formula (plain Dijkstra) at t = 256, and the
active-vertex count N_t at Time t against the same formula at t = 1024 for every level.
Weights are 0, so every count follows from first-passage times alone.
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


@pytest.mark.parametrize("j", [1, 2, 3, 4, 5])
def test_omega_small_equals_oracle(csp, j):
    inst = synth.fractal_environment(32, j)
    want = oracle.cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, labels=True)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True, phantoms=True)
    assert got.answer() == want.answer()
    assert (got.cycles, got.updates, got.launched) == (want.cycles, want.updates, want.launched)
    np.testing.assert_array_equal(got.trace, want.trace)
    assert got.phantoms == want.phantoms == 0
    np.testing.assert_array_equal(lat.labels(), want.labels.astype(np.int32))
    lat.close()


@pytest.mark.parametrize("j", [1, 4, 8])
def test_omega_trace_equals_first_passage(csp, j):
    inst = synth.fractal_environment(256, j)
    F1, X, tau, rows = brute.dijkstra_trace(inst.extents, inst.f1, inst.A, inst.B)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.solve(inst.A, inst.B, inst.M, trace=True)
    assert (got.F1, got.X, got.F2) == (F1, X, 0)
    np.testing.assert_array_equal(got.trace, rows)
    lat.close()


def test_omega_active_count_at_time_t(csp):
    t = 1024
    for j in range(1, 11):
        inst = synth.fractal_environment(t, j)
        tau = brute.tau(inst.extents, inst.f1, inst.A)
        want = brute.first_passage_row(inst.extents, inst.f1, tau, t)
        lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
        got = lat.solve(inst.A, inst.B, inst.M, trace=True, trace_cap=t + 8)
        lat.close()
        assert got.F1 == t + 1 and got.X == (inst.extents[1] - 1) * inst.extents[0] + t
        np.testing.assert_array_equal(got.trace[:, 0], np.arange(t + 2))
        assert tuple(int(x) for x in got.trace[t]) == want, j

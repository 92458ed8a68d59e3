"""GPU path reconstruction (csp_reconstruct_path, repeated application of Section 1)
against the oracle's reconstruction, and invariants on the full 128^3 cube."""
import numpy as np
import pytest

import oracle
from paper_1511_06441_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csp():
    from paper_1511_06441_gb300 import build, csp as mod
    build.build()
    return mod


def _path_sums(inst, path):
    """(F1, F2) of a path, reading each edge's weights straight from the SoA arrays."""
    st = synth.strides(inst.extents)
    V = inst.V
    f1 = inst.f1.reshape(-1).astype(np.int64)
    f2 = inst.f2.reshape(-1).astype(np.int64)
    t = w = 0
    for a, b in zip(path, path[1:]):
        lo, diff = min(a, b), abs(b - a)
        assert diff in st, (a, b)
        k = max(i for i, sk in enumerate(st) if sk == diff and inst.extents[i] > 1)  # (extent-1 axes repeat a stride)
        c = synth.coords(np.array([lo]), inst.extents)[0]
        assert c[k] + 1 < inst.extents[k] and f1[k * V + lo] > 0, (a, b)
        t += f1[k * V + lo]
        w += f2[k * V + lo]
    return int(t), int(w)


@pytest.mark.parametrize("seed", range(0, 40))
def test_tiny_paths_equal_oracle(csp, seed):
    inst = synth.random_small_instance(seed, max_vertices=20)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got = lat.reconstruct(inst.A, inst.B, inst.M)
    if want is None:
        assert got is None
    else:
        assert got.tolist() == want
    lat.close()


@pytest.mark.parametrize("ext,M", [([64, 64], 300), ([20, 20, 20], 260)])
def test_paths_equal_oracle(csp, ext, M):
    inst = synth.workload_64x64() if ext == [64, 64] else synth.workload_cube(ext[0], M)
    want, steps = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    r = lat.solve(inst.A, inst.B, M)
    got = lat.reconstruct(inst.A, inst.B, M, result=r)
    assert got.tolist() == want
    assert _path_sums(inst, want) == (r.F1, r.F2)
    lat.close()


def test_cube128_path_invariants(csp):
    inst = synth.workload_cube(128, 1600)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    r = lat.solve(inst.A, inst.B, 1600)
    path = lat.reconstruct(inst.A, inst.B, 1600, result=r)
    assert path[0] in set(inst.A.tolist()) and path[-1] == r.X
    assert len(set(path.tolist())) == len(path)
    assert _path_sums(inst, path.tolist()) == (r.F1, r.F2) and r.F2 < 1600
    lat.close()


# ---------------------------------------------------------------- one recorded solve + backtrack

@pytest.mark.parametrize("seed", range(0, 60))
def test_fast_path_equals_repeated_application_tiny(csp, seed):
    inst = synth.random_small_instance(seed, max_vertices=20)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got, r = lat.reconstruct_fast(inst.A, inst.B, inst.M)
    assert (got is None) == (want is None)
    if want is not None:
        assert got.tolist() == want
        assert _path_sums(inst, want) == (r.F1, r.F2)
    # first improvements only: either the same path or a refusal naming the missing record
    try:
        got1, _ = lat.reconstruct_fast(inst.A, inst.B, inst.M, log_capacity=-1)
        assert (got1 is None) == (want is None) and (want is None or got1.tolist() == want)
    except csp.CspError as e:
        assert e.status == csp.ERR_CAPACITY
    lat.close()


@pytest.mark.parametrize("ext,M", [([64, 64], 300), ([64, 64], 180), ([20, 20, 20], 260), ([20, 20, 20], 200)])
def test_fast_path_equals_repeated_application(csp, ext, M):
    inst = synth.workload_64x64() if ext == [64, 64] else synth.workload_cube(ext[0], M)
    want, _ = oracle.reconstruct(inst.extents, inst.f1, inst.f2, inst.A, inst.B, M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got, r = lat.reconstruct_fast(inst.A, inst.B, M)
    if want is None:
        assert got is None and r.F1 == -1
    else:
        assert got.tolist() == want
    lat.close()


@pytest.mark.parametrize("M", [800, 1600])
def test_fast_path_equals_gpu_repeated_application_cube128(csp, M):
    inst = synth.workload_cube(128, M)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    got, r = lat.reconstruct_fast(inst.A, inst.B, M)
    want = lat.reconstruct(inst.A, inst.B, M, result=r)
    assert got.tolist() == want.tolist()
    assert _path_sums(inst, got.tolist()) == (r.F1, r.F2)
    lat.close()


def test_fast_path_with_a_tiny_log_reports_capacity(csp):
    inst = synth.workload_cube(40, 500)
    lat = csp.Lattice(inst.extents, inst.f1, inst.f2)
    want, _ = lat.reconstruct_fast(inst.A, inst.B, 500)
    try:
        got, _ = lat.reconstruct_fast(inst.A, inst.B, 500, log_capacity=1)
        assert got.tolist() == want.tolist()
    except csp.CspError as e:
        assert e.status == csp.ERR_CAPACITY
    lat.close()

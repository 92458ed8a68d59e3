"""Batched mode: many instances in one persistent launch give, instance by instance,
exactly the results of separate csp_solve calls and of the oracle."""
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


def _mixed_instances(n, seed):
    out = []
    for i in range(n):
        r = synth.uniform_unit(seed, 900 + i, 4)
        if r[0] < 0.5:
            ext = [int(8 + r[1] * 60), int(6 + r[2] * 40)]
        else:
            ext = [int(4 + r[1] * 14)] * 3
        f1, f2 = synth.uniform_weights(ext, 1, 12, seed * 1000 + i)
        A = synth.face(ext, 0, 0)
        B = synth.face(ext, 0, ext[0] - 1)
        M = int(20 + r[3] * 12 * ext[0])
        out.append(synth.Instance(ext, f1, f2, A, B, M, f"mix{i}"))
    return out


def _answers(rs):
    return [(r.answer(), r.cycles, r.updates, r.launched) for r in rs]


@pytest.mark.parametrize("ctas,max_group", [(0, 0), (16, 8), (3, 2)])
def test_batch_equals_single_solves_and_oracle(csp, ctas, max_group):
    insts = _mixed_instances(40, 7)
    lats = [csp.Lattice(i.extents, i.f1, i.f2) for i in insts]
    items = [(L, i.A, i.B, i.M) for L, i in zip(lats, insts)]
    b = csp.Batch(items, ctas=ctas, max_group=max_group)
    b.run()
    got = b.results()
    assert all(r.status == csp.OK for r in got)
    single = [L.solve(i.A, i.B, i.M) for L, i in zip(lats, insts)]
    assert _answers(got) == _answers(single)
    for r, i in zip(got, insts):
        o = oracle.solve_instance(i, trace=False)
        assert (r.answer(), r.cycles, r.updates, r.launched) == (o.answer(), o.cycles, o.updates, o.launched)
    # a second run of the same captured graph gives the same results
    b.run()
    assert _answers(b.results()) == _answers(got)
    if max_group:
        assert b.schedule()["group"].max() >= 1
    b.close()


def test_batch_groups_of_several_ctas(csp):
    # few CTAs and big instances force groups > 1
    insts = [synth.workload_cube(24, 300 + 50 * k, seed=30 + k) for k in range(4)] + _mixed_instances(6, 11)
    lats = [csp.Lattice(i.extents, i.f1, i.f2) for i in insts]
    items = [(L, i.A, i.B, i.M) for L, i in zip(lats, insts)]
    b = csp.Batch(items, ctas=8, max_group=8)
    sched = b.schedule()
    assert sched["group"].max() > 1
    b.run()
    got = b.results()
    single = [L.solve(i.A, i.B, i.M) for L, i in zip(lats, insts)]
    assert _answers(got) == _answers(single)
    # the autotuner re-plans from the measured run; results stay identical
    b.tune(got)
    b.run()
    assert _answers(b.results()) == _answers(single)
    # direct launch without a graph
    nb = csp.Batch(items, ctas=8, max_group=8, no_graph=True)
    nb.run()
    assert _answers(nb.results()) == _answers(single)
    b.close()
    nb.close()


def test_batch_errors_are_per_instance(csp):
    insts = _mixed_instances(5, 3)
    lats = [csp.Lattice(i.extents, i.f1, i.f2) for i in insts]
    items = [(L, i.A, i.B, i.M) for L, i in zip(lats, insts)]
    items[2] = (lats[2], insts[2].A, insts[2].A[:1], insts[2].M)  # A and B overlap
    b = csp.Batch(items)
    b.run()
    got = b.results()
    assert got[2].status == csp.ERR_INVALID
    for k in (0, 1, 3, 4):
        assert got[k].status == csp.OK
        assert got[k].answer() == lats[k].solve(insts[k].A, insts[k].B, insts[k].M).answer()
    b.close()
    with pytest.raises(csp.CspError):
        csp.Batch([(lats[0], [], insts[0].B, 10)])


def test_solve_batch_retries_pool_overflow(csp):
    insts = [synth.workload_cube(20, 300, seed=5), synth.workload_64x64()]
    insts[1].M = 300
    lats = [csp.Lattice(i.extents, i.f1, i.f2) for i in insts]
    items = [(L, i.A, i.B, i.M) for L, i in zip(lats, insts)]
    b = csp.Batch(items, pool_capacity=256)
    b.run()
    assert csp.ERR_CAPACITY in [r.status for r in b.results()]
    b.close()
    got = csp.solve_batch(items, pool_capacity=256)
    assert all(r.status == csp.OK for r in got)
    assert [r.answer() for r in got] == [L.solve(i.A, i.B, i.M).answer() for L, i in zip(lats, insts)]

"""Serving mode: queries answered by the persistent server while others are in flight
give exactly the results they give alone (csp_solve), and the plain replay agrees."""
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


def _key(r):
    return (r.answer(), r.cycles, r.updates, r.launched)


@pytest.fixture(scope="module")
def setup(csp):
    ext, f1, f2 = synth.serving_lattice(side=10, d=4, seed=5)
    lat = csp.Lattice(ext, f1, f2)
    qs = synth.serving_queries(48, ext, seed=5)
    alone = [lat.solve(q.A, q.B, q.M) for q in qs]
    assert max(r.max_pool for r in alone) < 1 << 16  # fits the server's default slot pool
    # a query with an explicit (short) target list
    small = synth.Query(qs[0].A, qs[0].B[:50], qs[0].M)
    alone.append(lat.solve(small.A, small.B, small.M))
    qs.append(small)
    return ext, f1, f2, lat, qs, alone


def test_alone_equals_oracle(setup):
    ext, f1, f2, lat, qs, alone = setup
    for q, r in list(zip(qs, alone))[:12]:
        o = oracle.cycle(ext, f1, f2, q.A, q.B, q.M, trace=False)
        assert _key(r) == (o.answer(), o.cycles, o.updates, o.launched)


@pytest.mark.parametrize("group_ctas,max_groups", [(2, 4), (1, 6), (4, 3)])
def test_in_the_mix_equals_alone(csp, setup, group_ctas, max_groups):
    ext, f1, f2, lat, qs, alone = setup
    srv = csp.Server(lat, group_ctas=group_ctas, max_groups=max_groups, queue_capacity=16, session_seconds=120)
    # everything at once (admission limited by the ring), then a Poisson stream
    got, lat_s, mk = srv.replay(qs, np.zeros(len(qs)))
    assert [_key(r) for r in got] == [_key(r) for r in alone]
    assert all(r.status == csp.OK for r in got)
    got2, lat2, _ = srv.replay(qs, synth.poisson_arrivals(len(qs), 2000.0))
    assert [_key(r) for r in got2] == [_key(r) for r in alone]
    assert (lat2 > 0).all()
    # explicit target list (no hyperplane) through submit / poll
    t = srv.submit(qs[-1], use_hyperplane=False)
    r = None
    for _ in range(2000000):
        r = srv.poll(t)
        if r is not None:
            break
    assert r is not None and _key(r) == _key(alone[-1])
    srv.close()


def test_plain_replay_and_bad_queries(csp, setup):
    ext, f1, f2, lat, qs, alone = setup
    got, lat_s, mk = csp.plain_replay(lat, qs[:10], np.zeros(10))
    assert [_key(r) for r in got] == [_key(r) for r in alone[:10]]
    with pytest.raises(csp.CspError):  # more than 64 explicit targets
        srv0 = csp.Server(lat, group_ctas=1, max_groups=1, session_seconds=30)
        try:
            srv0.submit(qs[1], use_hyperplane=False)
        finally:
            srv0.close()
    srv = csp.Server(lat, group_ctas=1, max_groups=2, session_seconds=60)
    bad = synth.Query(np.arange(70, dtype=np.int64), qs[0].B, 100, qs[0].axis, qs[0].coord)  # more than 64 sources
    with pytest.raises(csp.CspError):
        srv.submit(bad)
    bad = synth.Query(qs[0].A, qs[0].B, 100, 7, 0)  # axis out of range
    with pytest.raises(csp.CspError):
        srv.submit(bad)
    srv.close()


@pytest.mark.parametrize("wide_depth", [2, 4, -1])
def test_wide_and_narrow_modes_give_the_alone_results(csp, setup, wide_depth):
    # a burst (the backlog switches the whole-grid mode to groups), then queries one at a time
    # with gaps (every group idle again: back to the whole grid), then another burst
    ext, f1, f2, lat, qs, alone = setup
    srv = csp.Server(lat, group_ctas=2, max_groups=4, queue_capacity=64, session_seconds=120, wide_depth=wide_depth)
    n = len(qs)
    arrivals = np.concatenate([np.zeros(n), 0.05 + 0.01 * np.arange(n), np.full(n, 0.05 + 0.01 * n + 0.05)])
    got, lat_s, mk = srv.replay(qs * 3, arrivals)
    assert [_key(r) for r in got] == [_key(r) for r in alone] * 3
    assert all(r.status == csp.OK for r in got)
    st = srv.stats()
    srv.close()
    assert st["wide_queries"] + st["narrow_queries"] == 3 * n
    if wide_depth > 0:
        assert st["wide_queries"] > 0 and st["narrow_queries"] > 0 and st["to_narrow"] >= 1 and st["to_wide"] >= 1
    else:
        assert st["wide_queries"] == 0 and st["to_wide"] == 0 and st["to_narrow"] == 0

"""The seeded input generator: determinism, ranges, layout, and the paper's edge counts."""
import json
import os

import numpy as np

from paper_1511_06441_gb300 import synth

FACTS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea & Flood 2014) output function applied to gamma*(i+1) + key
    def mix(z):
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 % 2**64
        z = (z ^ (z >> 27)) * 0x94D049BB133111EB % 2**64
        return z ^ (z >> 31)
    seed, stream = 7, 3
    key = mix((seed * 0x2545F4914F6CDD1D + stream) % 2**64)
    want = [mix((key + (i + 1) * 0x9E3779B97F4A7C15) % 2**64) for i in range(5)]
    assert synth.u64(seed, stream, 5).tolist() == want
    assert synth.u64(seed, stream, 3, offset=2).tolist() == want[2:]


def test_weights_layout_and_ranges():
    ext = [5, 4, 3]
    f1, f2 = synth.uniform_weights(ext, 1, 16, 2)
    assert f1.shape == (3, 60) and f1.dtype == np.uint8
    up = synth.upper_face_mask(ext)
    assert (f1[up] == 0).all() and (f2[up] == 0).all()
    assert f1[~up].min() >= 1 and f1[~up].max() <= 16
    f1b, _ = synth.uniform_weights(ext, 1, 16, 2)
    np.testing.assert_array_equal(f1, f1b)


def test_paper_cube_edge_counts():
    # the paper's table counts the undirected edges of n^3 cubes as 3 n^2 (n - 1)
    for n, V, E in FACTS["cube_edge_counts"]["cubes"]:
        ext = [n, n, n]
        assert synth.num_vertices(ext) == V
        up = synth.upper_face_mask(ext)
        assert int((~up).sum()) == E


def test_geometric_distribution():
    x = synth.geometric_clipped(3, 1, 200000, 1, 10, 255)
    assert x.min() == 1 and x.max() <= 255
    # P(X > k) = 0.9^k
    for k in (1, 5, 20):
        assert abs((x > k).mean() - 0.9 ** k) < 0.01
    f1, f2 = synth.anticorrelated_weights([64, 64])
    up = synth.upper_face_mask([64, 64])
    assert f1.dtype == np.uint16 and ((f1 + f2)[~up] == 256).all()


def test_workload_shapes():
    c1 = synth.workload_64x64()
    assert c1.V == 4096 and len(c1.A) == 64 and len(c1.B) == 64 and c1.M == 200
    assert int((~synth.upper_face_mask(c1.extents)).sum()) == 8064
    c2 = synth.workload_cube(16, 400)
    assert set(synth.coords(c2.A, c2.extents)[:, 0]) == {0}
    assert set(synth.coords(c2.B, c2.extents)[:, 0]) == {15}


def test_batch_and_queries():
    insts = synth.batch_instances(24)
    assert {i.d for i in insts} == {2, 3}
    for i in insts:
        assert not set(i.A.tolist()) & set(i.B.tolist())
        side = i.extents[0]
        assert 0.5 * side * 16 - 1 <= i.M <= 2 * side * 16
    ext = [6, 6, 6, 6]
    for q in synth.serving_queries(30, ext):
        assert 1 <= len(q.A) <= 64 and len(set(q.A.tolist())) == len(q.A)
        assert not set(q.A.tolist()) & set(q.B.tolist())
        assert 200 <= q.M <= 2000


def test_c_fill_equals_numpy_definition():
    for ext, lo, hi, dt in (([7, 5, 3], 1, 16, np.uint8), ([33, 17], 0, 300, np.uint16), ([4, 3, 3, 2], 1, 20, np.uint8)):
        a1, a2 = synth.uniform_weights(ext, lo, hi, 11, dtype=dt, use_c=True)
        b1, b2 = synth.uniform_weights(ext, lo, hi, 11, dtype=dt, use_c=False)
        np.testing.assert_array_equal(a1, b1)
        np.testing.assert_array_equal(a2, b2)


def test_face_matches_coordinates():
    ext = [5, 4, 3]
    for k in range(3):
        for c in (0, ext[k] - 1):
            want = np.nonzero(synth.coords(np.arange(60), ext)[:, k] == c)[0]
            np.testing.assert_array_equal(synth.face(ext, k, c), want)


def test_point_source_workload():
    inst = synth.workload_point_source(16, seed=6)
    assert inst.A.tolist() == [8 + 8 * 16]
    assert sorted(inst.B.tolist()) == [0, 15, 240, 255]
    assert inst.f1.dtype == np.uint8 and 1 <= inst.f1[0, 0] <= 16

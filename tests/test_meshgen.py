"""Seeded input generators: sizes, determinism, conformity of the synthetic meshes."""
import numpy as np

from paper_1401_3301_gb300 import meshgen


def test_counts_and_determinism():
    m = meshgen.square_mesh(100, seed=0)
    assert (m.nq, m.nme) == (10201, 20000)
    m2 = meshgen.square_mesh(100, seed=0)
    np.testing.assert_array_equal(m.q, m2.q)
    np.testing.assert_array_equal(m.me, m2.me)
    k = meshgen.kuhn_cube_mesh(8, seed=3)
    assert (k.nq, k.nme) == (9 ** 3, 6 * 8 ** 3)
    assert k.me.dtype == np.int32 and k.q.dtype == np.float64
    assert k.me.min() == 0 and k.me.max() == k.nq - 1


def test_kuhn_conforming_and_oriented_both_ways():
    k = meshgen.kuhn_cube_mesh(6, seed=1, jitter=0.15)
    X = k.q[:, k.me]  # (3, 4, nme)
    B = X[:, 1:, :] - X[:, :1, :]
    det = np.linalg.det(np.moveaxis(B, 2, 0))
    h = 1.0 / 6
    assert np.abs(det).min() >= 0.1 * h ** 3 * 0.999
    assert (det > 0).sum() == (det < 0).sum()  # half the Kuhn tets are negatively oriented
    assert abs(np.abs(det).sum() / 6 - 1.0) < 1e-12  # they tile the unit cube
    # every interior face is shared by exactly two tets
    faces = {}
    for e in range(k.nme):
        v = k.me[:, e]
        for drop in range(4):
            f = tuple(sorted(np.delete(v, drop)))
            faces[f] = faces.get(f, 0) + 1
    assert max(faces.values()) == 2


def test_streams_are_independent_and_uniform():
    a = meshgen.uniform(meshgen.stream_key(0, 1), 100000)
    b = meshgen.uniform(meshgen.stream_key(0, 2), 100000)
    assert 0.49 < a.mean() < 0.51 and a.min() >= 0 and a.max() < 1
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    g = meshgen.normal(meshgen.stream_key(0, 4), 100000)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1) < 0.02
    p = meshgen.permutation(meshgen.stream_key(0, 2), 1000)
    assert sorted(p.tolist()) == list(range(1000))
    s = meshgen.batch_sizes(0, 256, 16, 512)
    assert s.min() >= 16 and s.max() <= 512

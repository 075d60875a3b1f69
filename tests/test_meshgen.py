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


def test_recipe_sizes_of_the_other_workloads():
    # P_k lattice meshes: (kN + 1)^d nodes, the coarse element count, ndfe rows
    for d, N, k in ((2, 5, 3), (3, 3, 2)):
        m = meshgen.pk_mesh(d, N, k, seed=1)
        ndfe = {(2, 3): 10, (3, 2): 10}[(d, k)]
        assert m.nq == (k * N + 1) ** d and m.me.shape == (ndfe, (2 if d == 2 else 6) * N ** d)
        assert m.me.min() == 0 and m.me.max() == m.nq - 1
    # the facet workload: 2 N^2 triangles in 3D on (N+1)^2 vertices
    s = meshgen.surface_mesh(20, seed=0)
    assert s.q.shape == (3, 21 ** 2) and s.me.shape == (3, 2 * 20 ** 2)
    # boundary of the Kuhn cube: 2 N^2 triangles on each of the 6 faces
    k = meshgen.kuhn_cube_mesh(5, seed=2)
    assert meshgen.boundary_facets(k).shape == (3, 12 * 5 ** 2)
    # general-operator records: d*d + 2d + 1 values; A = exp(g0) I + 0.3 N is not symmetric
    # and its symmetric part is positive definite for most records; a0 = exp(g1) > 0
    c = meshgen.general_coefficients(3, 3, 2000)
    assert c.shape == (2000, 16)
    A = c[:, :9].reshape(-1, 3, 3)
    assert np.abs(A - A.transpose(0, 2, 1)).max(axis=(1, 2)).min() > 0
    sym = 0.5 * (A + A.transpose(0, 2, 1))
    assert (np.linalg.eigvalsh(sym).min(axis=1) > 0).mean() > 0.7 and (c[:, 15] > 0).all()

"""Seeded synthetic inputs: simplicial meshes, coefficient fields and random vectors.

This module only produces input data. It holds none of the assembly arithmetic
(no volumes, gradients or element matrices), so both the CUDA path and the FP64
oracle can be fed from it.

Layout follows the mesh data structure of the paper (Section 2, Table 1):
``q`` is a d-by-nq array of vertex coordinates and ``me`` a (d+1)-by-nme
connectivity array. Here both are C-contiguous "structure of arrays" numpy
arrays: ``q[c, v]`` is coordinate c of vertex v (float64), ``me[a, k]`` is the
0-based vertex index of local vertex a of element k (int32). The paper's
arrays are 1-based; subtract 1 at any Matlab-style boundary.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value i
of a stream with key s is mix(s + (i+1) * 0x9E3779B97F4A7C15). One stream per
purpose, so changing one input never shifts another.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream purposes
JITTER, ELEM_PERM, VERT_PERM, VERT_WEIGHT, ELEM_WEIGHT, VECTORS, BATCH_SIZES, GEN_COEF, SHAPES = (
    1, 2, 3, 4, 5, 6, 7, 8, 9)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, purpose: int) -> int:
    """Key of the stream for (seed, purpose): one splitmix64 step of a packed word."""
    z = np.array([(int(seed) * 0x100 + int(purpose)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
    return int(_mix(z)[0])


def splitmix64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset..offset+n-1 of the counter-based splitmix64 stream ``key``."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + i * _GOLDEN
    return _mix(z)


def uniform(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(key, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: int, n: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(key, 2 * m)
    u1, u2 = 1.0 - u[0::2], u[1::2]  # u1 in (0, 1]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def permutation(key: int, n: int) -> np.ndarray:
    """A random permutation of 0..n-1 (stable argsort of 64-bit random keys)."""
    return np.argsort(splitmix64(key, n), kind="stable").astype(np.int64)


@dataclass
class Mesh:
    d: int
    q: np.ndarray   # (d, nq) float64
    me: np.ndarray  # (d+1, nme) int32, 0-based

    @property
    def nq(self) -> int:
        return int(self.q.shape[1])

    @property
    def nme(self) -> int:
        return int(self.me.shape[1])


def _finish(d, q, me, seed, jitter, interior, h, perm_vertices, perm_elements):
    if jitter > 0.0:
        idx = np.nonzero(interior)[0]
        u = uniform(stream_key(seed, JITTER), d * idx.size).reshape(d, idx.size)
        q[:, idx] += (2.0 * u - 1.0) * (jitter * h)
    if perm_vertices:
        new_of_old = permutation(stream_key(seed, VERT_PERM), q.shape[1])
        qn = np.empty_like(q)
        qn[:, new_of_old] = q
        q = qn
        me = new_of_old[me].astype(np.int32)
    if perm_elements:
        p = permutation(stream_key(seed, ELEM_PERM), me.shape[1])
        me = me[:, p]
    return Mesh(d, np.ascontiguousarray(q), np.ascontiguousarray(me, dtype=np.int32))


def square_mesh(N: int, seed: int = 0, jitter: float = 0.2, perm_vertices: bool = True,
                perm_elements: bool = True) -> Mesh:
    """Unit square, N x N cells, each split into 2 triangles along the (0,0)-(1,1) diagonal.

    (N+1)^2 vertices, 2 N^2 triangles; interior vertices moved by U(-jitter h, jitter h)
    per coordinate (h = 1/N); optional random vertex relabelling and element order.
    """
    n1 = N + 1
    j, i = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    q = np.stack([i.ravel() / N, j.ravel() / N]).astype(np.float64)
    interior = ((i > 0) & (i < N) & (j > 0) & (j < N)).ravel()
    cj, ci = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    v00 = (cj * n1 + ci).ravel()
    v10, v01 = v00 + 1, v00 + n1
    v11 = v01 + 1
    t1 = np.stack([v00, v10, v11])
    t2 = np.stack([v00, v11, v01])
    me = np.stack([t1, t2], axis=2).reshape(3, -1).astype(np.int32)
    return _finish(2, q, me, seed, jitter, interior, 1.0 / N, perm_vertices, perm_elements)


_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def kuhn_cube_mesh(N: int, seed: int = 0, jitter: float = 0.15, perm_vertices: bool = False,
                   perm_elements: bool = True) -> Mesh:
    """Unit cube, N^3 cells, each split into the 6 Kuhn tetrahedra around its main diagonal.

    Vertex (i, j, k) has index (k (N+1) + j)(N+1) + i. Tetrahedron sigma of a cell is the
    monotone lattice path c000 -> +e_s0 -> +e_s1 -> c111; half of them are negatively
    oriented. Interior vertices are moved by U(-jitter h, jitter h) per coordinate.
    """
    n1 = N + 1
    k, j, i = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    q = np.stack([i.ravel() / N, j.ravel() / N, k.ravel() / N]).astype(np.float64)
    interior = ((i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)).ravel()
    ck, cj, ci = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    base = ((ck * n1 + cj) * n1 + ci).ravel().astype(np.int64)
    step = (1, n1, n1 * n1)
    tets = []
    for s in _KUHN_PERMS:
        p1 = base + step[s[0]]
        p2 = p1 + step[s[1]]
        p3 = base + 1 + n1 + n1 * n1
        tets.append(np.stack([base, p1, p2, p3]))
    me = np.stack(tets, axis=2).reshape(4, -1).astype(np.int32)
    return _finish(3, q, me, seed, jitter, interior, 1.0 / N, perm_vertices, perm_elements)


def _rotation(key: int, i: int, d: int) -> np.ndarray:
    """A random d x d rotation (QR of a Gaussian matrix, signs fixed, det +1)."""
    u = uniform(key, 2 * d * d, offset=2 * d * d * i)
    g = np.sqrt(-2.0 * np.log(1.0 - u[0::2])) * np.cos(2.0 * np.pi * u[1::2])
    Q, R = np.linalg.qr(g.reshape(d, d))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def badly_shaped_mesh(d: int, flat: list, seed: int = 0, size: float = 0.02,
                      center=None, spread: float = 0.1) -> Mesh:
    """Isolated, badly shaped simplices (no shared vertices), three per flatness value eps
    in ``flat``, each turned by its own random rotation, scaled to ``size`` and placed at a
    random point of the box of side ``spread`` around ``center`` (default the middle of the
    unit box; the default spread of 5 sizes is the extent of an element chunk of a mesh). 3D: a sliver (four nearly coplanar vertices spanning a unit square, lifted by
    -+eps), a cap (one vertex at height eps over the middle of the opposite face) and a
    needle (three edges along one direction, spread by eps); det B is about eps (eps^2 for
    the needle) of the products it is formed from. 2D: a cap (one vertex at height eps over
    the middle of the opposite edge), a needle (a short edge of length eps) and a sliver
    (the cap's apex moved near an end of the base)."""
    key = stream_key(seed, SHAPES)
    c0 = np.full(d, 0.5) if center is None else np.asarray(center, dtype=np.float64)
    verts, k = [], 0
    for eps in flat:
        if d == 3:
            shapes = [
                [(0, 0, eps), (1, 0, -eps), (1, 1, eps), (0, 1, -eps)],                # sliver
                [(0, 0, 0), (1, 0, 0), (0.3, 0.9, 0), (0.45, 0.3, eps)],            # cap
                [(0, 0, 0), (1, 0, 0), (0.6, np.sqrt(eps), 0), (0.4, 0, np.sqrt(eps))],  # needle
            ]
        else:
            shapes = [[(0, 0), (1, 0), (0.5, eps)], [(0, 0), (eps, 0), (0.3, 1.0)], [(0, 0), (1, 0), (0.98, eps)]]
        for sh in shapes:
            X = np.array(sh, dtype=np.float64)
            X = X - X.mean(axis=0)
            R = _rotation(key, k, d)
            off = (uniform(key, d, offset=10 ** 6 + d * k) - 0.5) * spread
            verts.append((X @ R.T) * size + c0 + off)
            k += 1
    q = np.concatenate(verts, axis=0).T.copy()
    me = np.arange(q.shape[1], dtype=np.int32).reshape(-1, d + 1).T.copy()
    return Mesh(d, q, me)


def pk_node_order(d: int, k: int) -> list:
    """Local node order of a P_k simplex (App. D) as multi-indices alpha, |alpha| = k: the
    d+1 vertices k e_0, ..., k e_d first, then the other multi-indices in lexicographically
    decreasing order."""
    verts = [tuple(k if i == j else 0 for i in range(d + 1)) for j in range(d + 1)]
    out = list(verts)
    def rec(prefix, left, slots):
        if slots == 1:
            yield prefix + (left,)
            return
        for x in range(left, -1, -1):
            yield from rec(prefix + (x,), left - x, slots - 1)
    out += [a for a in rec((), k, d + 1) if a not in verts]
    return out


def pk_mesh(d: int, N: int, k: int, seed: int = 0, jitter: float | None = None, perm_nodes: bool = False,
            perm_elements: bool = True) -> Mesh:
    """P_k mesh (App. D) of the unit square (d=2) or the Kuhn cube (d=3) with N cells per side.

    The simplices are unimodular, so their P_k nodes are exactly the points of the k-times
    finer lattice: (kN+1)^d nodes, numbered like the coarse vertices on the fine lattice.
    me is (ndfe, nme), rows in pk_node_order(d, k). Node coordinates are the affine images
    sum_i alpha_i x_i / k of the jittered coarse vertices, taken from the first element
    (in generation order) holding the node. k = 1 gives the P1 mesh with the same jitter.
    """
    if jitter is None:
        jitter = 0.2 if d == 2 else 0.15
    base = (square_mesh if d == 2 else kuhn_cube_mesh)(N, seed=seed, jitter=jitter, perm_vertices=False,
                                                       perm_elements=False)
    n1, f1 = N + 1, k * N + 1
    vid = np.arange(base.nq)
    ic = np.stack([(vid // n1 ** c) % n1 for c in range(d)])            # coarse integer coordinates
    alphas = np.array(pk_node_order(d, k), dtype=np.int64)              # (ndfe, d+1)
    corner = ic[:, base.me]                                             # (d, d+1, nme)
    fine = np.einsum("ai,cie->ace", alphas, corner)                     # (ndfe, d, nme)
    ids = np.zeros((alphas.shape[0], base.nme), dtype=np.int64)
    for c in range(d):
        ids += fine[:, c, :] * f1 ** c
    xc = base.q[:, base.me]                                             # (d, d+1, nme)
    xf = np.einsum("ai,cie->ace", alphas.astype(np.float64), xc) / k    # (ndfe, d, nme)
    flat_ids = ids.T.ravel()                                            # element-major, first = lowest element
    _, first = np.unique(flat_ids, return_index=True)
    q = np.empty((d, f1 ** d))
    q[:, flat_ids[first]] = xf.transpose(1, 2, 0).reshape(d, -1)[:, first]
    me = ids
    if perm_nodes:
        new_of_old = permutation(stream_key(seed, VERT_PERM), q.shape[1])
        qn = np.empty_like(q)
        qn[:, new_of_old] = q
        q, me = qn, new_of_old[me]
    if perm_elements:
        me = me[:, permutation(stream_key(seed, ELEM_PERM), me.shape[1])]
    return Mesh(d, np.ascontiguousarray(q), np.ascontiguousarray(me, dtype=np.int32))


def surface_mesh(N: int, seed: int = 0) -> Mesh:
    """A triangulated surface in 3D: the jittered, permuted unit-square mesh of
    square_mesh(N) lifted to the height field z = 0.25 sin(2 pi x) cos(2 pi y). Returns
    Mesh(d=3, q (3, nq), me (3, ntriangles)), a facet mesh for boundary operators."""
    m = square_mesh(N, seed=seed)
    z = 0.25 * np.sin(2.0 * np.pi * m.q[0]) * np.cos(2.0 * np.pi * m.q[1])
    return Mesh(3, np.ascontiguousarray(np.vstack([m.q, z[None, :]])), m.me)


def boundary_facets(mesh: Mesh) -> np.ndarray:
    """Facets (d-1 simplices) that belong to exactly one element: (d, nfacets) int32,
    vertex indices into the same q, in the order of first appearance."""
    d, me = mesh.d, mesh.me
    faces = np.concatenate([np.delete(me, drop, axis=0) for drop in range(d + 1)], axis=1).T
    key = np.sort(faces, axis=1)
    _, first, counts = np.unique(key, axis=0, return_index=True, return_counts=True)
    keep = np.sort(first[counts == 1])
    return np.ascontiguousarray(faces[keep].T.astype(np.int32))


def vertex_weights(seed: int, nq: int) -> np.ndarray:
    """Per-vertex weight w = exp(g), g ~ N(0, 1) iid."""
    return np.exp(normal(stream_key(seed, VERT_WEIGHT), nq))


def element_weights(seed: int, nme: int) -> np.ndarray:
    """Per-element lognormal(0, 1) coefficient."""
    return np.exp(normal(stream_key(seed, ELEM_WEIGHT), nme))


def general_coefficients(seed: int, d: int, n: int) -> np.ndarray:
    """n records (rows) of convection-diffusion-reaction coefficients, (n, d*d + 2d + 1):
    A = exp(g0) I + 0.3 N (a non-symmetric tensor, row-major; its symmetric part is positive
    definite for most records), b and c
    with N(0, 1) entries, a0 = exp(g1); g0, g1 and the entries of N iid N(0, 1)."""
    nc = d * d + 2 * d + 1
    z = normal(stream_key(seed, GEN_COEF), (nc + 2) * n).reshape(n, nc + 2)
    out = np.empty((n, nc))
    out[:, : d * d] = 0.3 * z[:, : d * d]
    out[:, 0 : d * d : d + 1] += np.exp(z[:, nc : nc + 1])
    out[:, d * d : nc - 1] = z[:, d * d : nc - 1]
    out[:, nc - 1] = np.exp(z[:, nc + 1])
    return out


def random_vectors(seed: int, n: int, count: int = 2) -> np.ndarray:
    """``count`` iid N(0, 1) vectors of length n (rows)."""
    return normal(stream_key(seed, VECTORS), count * n).reshape(count, n)


def batch_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """``count`` integers uniform in [lo, hi]."""
    z = splitmix64(stream_key(seed, BATCH_SIZES), count)
    return (lo + (z % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def lame_from_young(E: float, nu: float) -> tuple[float, float]:
    """Isotropic Lame parameters (lambda, mu) from Young's modulus and Poisson ratio (3D)."""
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))

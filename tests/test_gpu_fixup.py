"""GPU parity of the fixup pass (the shared entries of FE_REASM_CHUNKED) on long lists of
partial sums.

A fan of K = 20 elements around one vertex (2D) or one edge (3D), each element placed at
the head of its own 32-element chunk (input order kept; the rest of each chunk is a
disjoint padding mesh), puts that vertex or edge in 20 chunks: its fixup sums 20 partials,
past the four each thread loads ahead. Values are checked against the FP64 oracle in all
three forms.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

K, CHUNK = 20, 32


def fan_mesh(d: int) -> meshgen.Mesh:
    t = 2 * math.pi * np.arange(K) / K
    i = np.arange(K)
    if d == 2:  # hub vertex 0, ring 1..K
        q = np.concatenate([np.zeros((2, 1)), np.stack([np.cos(t), np.sin(t)])], axis=1)
        fan = np.stack([np.zeros(K, dtype=np.int64), 1 + i, 1 + (i + 1) % K])
        pad, scale = meshgen.square_mesh(18, seed=5, perm_elements=False), 3.0
    else:  # hub edge (0, 1) along z, ring 2..K+1
        ring = np.stack([np.cos(t), np.sin(t), np.zeros(K)])
        q = np.concatenate([np.array([[0.0, 0.0], [0.0, 0.0], [-1.0, 1.0]]), ring], axis=1)
        fan = np.stack([np.zeros(K, dtype=np.int64), np.ones(K, dtype=np.int64), 2 + i, 2 + (i + 1) % K])
        pad, scale = meshgen.kuhn_cube_mesh(5, seed=5, perm_elements=False), 2.0
    # disjoint from the fan, and with elements not much smaller than the extent of a chunk
    # (the F64X form's coordinates are taken relative to a vertex of the chunk)
    qp = pad.q * scale
    qp[0] += 1.5
    mp = pad.me.astype(np.int64) + q.shape[1]
    assert mp.shape[1] >= (CHUNK - 1) * K
    cols = []
    for k in range(K):  # fan element k heads chunk k
        cols += [fan[:, k:k + 1], mp[:, (CHUNK - 1) * k:(CHUNK - 1) * (k + 1)]]
    cols.append(mp[:, (CHUNK - 1) * K:])
    return meshgen.Mesh(d, np.concatenate([q, qp], axis=1), np.concatenate(cols, axis=1).astype(np.int32))


def chunks_per_entity(me, size):
    """Number of distinct chunks each vertex (size 1) or edge (size 2) lies in."""
    ch = np.arange(me.shape[1]) // CHUNK
    nv = me.shape[0]
    if size == 1:
        ent = [me[a].astype(np.int64) for a in range(nv)]
    else:
        ent = [np.minimum(me[a], me[b]).astype(np.int64) * (1 << 32) + np.maximum(me[a], me[b])
               for a in range(nv) for b in range(a + 1, nv)]
    pairs = np.unique(np.stack([np.concatenate(ent), np.tile(ch, len(ent))]), axis=1)
    _, counts = np.unique(pairs[0], return_counts=True)
    return counts


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_fan_long_partial_lists(d, prec):
    fe = fe_or_skip()
    m = fan_mesh(d)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_KEEP_ORDER | fe.PATTERN_CHUNK(CHUNK))
    info = p.plan_info()
    assert info["chunk"] == CHUNK
    # the plan's shared entities and partial sums, against a count of the distinct chunks
    # each vertex and edge lies in (the input order is kept: chunk = element // CHUNK)
    for kind, cnt in (("vertices", chunks_per_entity(m.me, 1)), ("edges", chunks_per_entity(m.me, 2))):
        sh = cnt[cnt >= 2]
        assert (info["shared_" + kind], info["partial_" + kind]) == (sh.size, int(sh.sum())), kind
    assert chunks_per_entity(m.me, d - 1).max() == K  # the hub vertex (2D) or edge (3D)
    for kind, ref in (("mass", oracle.assemble(oracle.MASS, m.q, m.me)),
                      ("stiff", oracle.assemble(oracle.STIFF, m.q, m.me))):
        vals = (fe.fe_assemble_mass if kind == "mass" else fe.fe_assemble_stiff)(p, q, prec=prec)
        assert p.status() == (0, -1)
        check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D fan {kind}, chunk {CHUNK}")

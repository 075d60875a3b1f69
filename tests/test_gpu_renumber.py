"""Morton vertex renumbering utility: the order matches a NumPy computation of the same
Morton codes bit for bit, the renumbered mesh is the permuted mesh, and its stiffness
matrix is the permuted matrix."""
import numpy as np
import pytest

from paper_1401_3301_gb300 import meshgen
from helpers import fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def morton_order_reference(q, qbits=21):
    d, nq = q.shape
    lo, hi = q.min(axis=1), q.max(axis=1)
    t = np.clip((q - lo[:, None]) / (hi - lo)[:, None], 0.0, 1.0)
    iq = np.minimum((t * float(1 << qbits)).astype(np.uint64), np.uint64((1 << qbits) - 1))
    code = np.zeros(nq, dtype=np.uint64)
    for c in range(d):
        for b in range(qbits):
            code |= ((iq[c] >> np.uint64(b)) & np.uint64(1)) << np.uint64(b * d + c)
    return np.argsort(code, kind="stable").astype(np.int32)


@pytest.mark.parametrize("d,N", [(2, 40), (3, 12)])
def test_order_and_renumbered_mesh(d, N):
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(N, seed=50) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=50, perm_vertices=True)
    q, me = to_cuda(m.q), to_cuda(m.me)
    order = fe.fe_morton_vertex_order(q)
    ref = morton_order_reference(m.q)
    np.testing.assert_array_equal(order.cpu().numpy(), ref)
    q2, me2 = fe.fe_apply_vertex_order(q, me, order)
    inv = np.empty_like(ref)
    inv[ref] = np.arange(ref.size, dtype=np.int32)
    np.testing.assert_array_equal(q2.cpu().numpy(), m.q[:, ref])
    np.testing.assert_array_equal(me2.cpu().numpy(), inv[m.me])
    # same matrix up to the permutation, value for value
    p1, p2 = fe.fe_pattern(q, me), fe.fe_pattern(q2, me2)
    a1, a2 = fe.fe_assemble_stiff(p1, q), fe.fe_assemble_stiff(p2, q2)
    rp1, ci1 = (t.cpu().numpy() for t in p1.csr())
    rp2, ci2 = (t.cpu().numpy() for t in p2.csr())
    r1 = np.repeat(np.arange(m.nq), np.diff(rp1))
    r2 = np.repeat(np.arange(m.nq), np.diff(rp2))
    k1 = inv[r1].astype(np.int64) * m.nq + inv[ci1]
    k2 = r2.astype(np.int64) * m.nq + ci2
    o1, o2 = np.argsort(k1), np.argsort(k2)
    np.testing.assert_array_equal(k1[o1], k2[o2])
    np.testing.assert_allclose(a1.cpu().numpy()[o1], a2.cpu().numpy()[o2], rtol=1e-14, atol=1e-15)


def test_rejects_a_bad_order():
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(5, seed=51)
    q, me = to_cuda(m.q), to_cuda(m.me)
    bad = torch.arange(m.nq, dtype=torch.int32, device="cuda")
    bad[3] = m.nq + 7
    with pytest.raises(fe.FEError):
        fe.fe_apply_vertex_order(q, me, bad)

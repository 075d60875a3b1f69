"""Edge cases of the boundary: the smallest meshes, unreferenced vertices (empty rows),
size limits caught before any device work, degenerate elements in every operator, and
results that do not depend on the launch configuration."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def test_single_element_2d_and_3d():
    fe = fe_or_skip()
    for X in (np.array([[0.0, 1.0, 0.2], [0.0, 0.1, 1.0]]), np.array([[0.0, 1.0, 0.0, 0.1], [0.0, 0.0, 1.0, 0.2],
                                                                      [0.0, 0.1, 0.0, 1.0]])):
        d = X.shape[0]
        me = np.arange(d + 1, dtype=np.int32).reshape(d + 1, 1)
        p = fe.fe_pattern(to_cuda(X), to_cuda(me))
        assert p.nnz == (d + 1) ** 2
        for kind, fn in ((oracle.MASS, fe.fe_assemble_mass), (oracle.STIFF, fe.fe_assemble_stiff)):
            ref = oracle.assemble(kind, X, me)
            for prec in (0, 1):
                got = fn(p, to_cuda(X), prec=prec).double().cpu().numpy()
                check_values(got, ref, prec, "single element")


def test_unreferenced_vertices_give_empty_rows():
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(4, seed=11)
    extra = np.random.default_rng(12).random((3, 5))
    q = np.concatenate([m.q[:, :40], extra, m.q[:, 40:]], axis=1)   # five vertices no element uses
    me = np.where(m.me >= 40, m.me + 5, m.me).astype(np.int32)
    ref = oracle.assemble(oracle.STIFF, q, me)
    p = fe.fe_pattern(to_cuda(q), to_cuda(me))
    rp, ci = (t.cpu().numpy() for t in p.csr())
    np.testing.assert_array_equal(rp.astype(np.int64), ref["row_ptr"])
    assert np.all(np.diff(rp)[40:45] == 0)
    for strategy in (0, 1, 2):
        p.set_strategy(strategy)
        got = fe.fe_assemble_stiff(p, to_cuda(q)).cpu().numpy()
        check_values(got, ref, 0, "3D stiffness, unreferenced vertices")


def test_size_limits_are_checked_before_any_device_work():
    fe = fe_or_skip()
    L = fe.lib()

    class Mesh(C.Structure):
        _fields_ = [("d", C.c_int32), ("nq", C.c_int64), ("nme", C.c_int64), ("q", C.c_void_p), ("me", C.c_void_p)]

    h = C.c_void_p()
    dummy = C.c_void_p(16)  # never dereferenced: the counts are rejected first
    # nme (d+1)^2 slots beyond int32
    rc = L.fe_pattern(C.byref(Mesh(3, 1000, (1 << 31) // 16 + 1, dummy, dummy)), 1, 0, None, C.byref(h))
    assert rc == 4  # FE_ERR_OVERFLOW
    # m * nq beyond int32
    rc = L.fe_pattern(C.byref(Mesh(3, (1 << 31) // 3 + 1, 10, dummy, dummy)), 3, 0, None, C.byref(h))
    assert rc == 4
    # empty meshes and bad dimensions are argument errors
    assert L.fe_pattern(C.byref(Mesh(3, 10, 0, dummy, dummy)), 1, 0, None, C.byref(h)) == 1
    assert L.fe_pattern(C.byref(Mesh(4, 10, 10, dummy, dummy)), 1, 0, None, C.byref(h)) == 1


def test_degenerate_elements_are_reported_by_every_operator():
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(4, seed=13)
    qb = m.q.copy()
    a, b = m.me[0, 7], m.me[1, 7]
    qb[:, b] = qb[:, a]  # collapse an edge: every element holding both vertices is flat
    q, me = to_cuda(qb), to_cuda(m.me)
    p, pv = fe.fe_pattern(q, me), fe.fe_pattern(q, me, m=3)
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    cf = to_cuda(meshgen.general_coefficients(1, 3, m.nme))
    u = torch.ones(m.nq, dtype=torch.float64, device="cuda")
    dq = torch.empty((3, m.nq), dtype=torch.float64, device="cuda")
    calls = [lambda: fe.fe_assemble_mass(p, q), lambda: fe.fe_assemble_stiff(p, q),
             lambda: fe.fe_assemble_stiff(p, q, prec=fe.F32), lambda: fe.fe_assemble_stiff(p, q, prec=fe.F64X),
             lambda: fe.fe_assemble_mass(p, q, prec=fe.F64X),
             lambda: fe.fe_assemble_general(p, q, cf, fe.COEF_P0),
             lambda: fe.fe_assemble_general(p, q, cf, fe.COEF_P0, prec=fe.F64X)]
    for prec in (fe.F64, fe.F64X):
        calls.append(lambda prec=prec: fe.fe_assemble_stiff_backward(p, q, None, fe.COEF_NONE, u, u, None, None, dq,
                                                                     prec=prec))
    for call in calls:
        call()
        code, eid = p.status()
        assert code == 3 and 0 <= eid < m.nme
        assert a in m.me[:, eid] and b in m.me[:, eid]
    for prec in (fe.F64, fe.F32, fe.F64X):
        T = torch.float32 if prec == fe.F32 else torch.float64
        fe.fe_assemble_elas(pv, q, one.to(T), fe.COEF_SCALAR, one.to(T), fe.COEF_SCALAR, prec=prec)
        code, eid = pv.status()
        assert code == 3 and a in m.me[:, eid] and b in m.me[:, eid], prec
    assert p.status() == (0, -1)  # read and cleared


@pytest.mark.parametrize("prec", [0, 1])
def test_values_do_not_depend_on_threads_per_block(prec):
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(10, seed=14)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    out = []
    for t in (128, 256, 512):
        p.set_threads(t)
        out.append(fe.fe_assemble_stiff(p, q, prec=prec))
    assert torch.equal(out[0], out[1]) and torch.equal(out[1], out[2])


def test_nan_coordinate_is_reported_as_degenerate():
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(4, seed=15)
    qb = m.q.copy()
    v = m.me[2, 20]
    qb[1, v] = np.nan
    q, me = to_cuda(qb), to_cuda(m.me)
    p = fe.fe_pattern(q, me)  # the pattern does not read coordinates' values for its indices
    for prec in (fe.F64, fe.F32, fe.F64X):
        fe.fe_assemble_stiff(p, q, prec=prec)
        code, eid = p.status()
        assert code == 3 and v in m.me[:, eid], prec
    # a facet mesh with a NaN on one of its vertices
    fa = meshgen.boundary_facets(m)
    qf = m.q.copy()
    vf = fa[1, 5]
    qf[0, vf] = np.nan
    pb = fe.fe_boundary_pattern(to_cuda(qf), to_cuda(fa))
    for prec in (fe.F64, fe.F32, fe.F64X):
        fe.fe_assemble_mass(pb, to_cuda(qf), prec=prec)
        code, eid = pb.status()
        assert code == 3 and vf in fa[:, eid], prec

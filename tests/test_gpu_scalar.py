"""GPU parity of the scalar operators (mass, weighted mass, stiffness) through the C ABI.

Every case compares the CUDA path with the FP64 oracle on the same seeded inputs:
the CSR pattern bit for bit, values within 1e-12 (FP64 form) or 1e-5 (FP32 form)
of the normalised per-nonzero error.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

def mesh(d, N, seed=0):
    return meshgen.square_mesh(N, seed=seed) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=seed)


def run(fe, p, kind, q, prec, coef=None):
    import torch
    T = torch.float64 if prec == 0 else torch.float32
    if kind == "mass":
        return fe.fe_assemble_mass(p, q, prec=prec)
    if kind == "wmass_p1":
        return fe.fe_assemble_wmass(p, q, coef.to(T), fe.COEF_P1, prec=prec)
    if kind == "wmass_p0":
        return fe.fe_assemble_wmass(p, q, coef.to(T), fe.COEF_P0, prec=prec)
    if kind == "stiff":
        return fe.fe_assemble_stiff(p, q, prec=prec)
    if kind == "stiff_w":
        return fe.fe_assemble_stiff(p, q, coef.to(T), fe.COEF_P0, prec=prec)
    raise ValueError(kind)


def oracle_ref(kind, m, coef):
    if kind == "mass":
        return oracle.assemble(oracle.MASS, m.q, m.me)
    if kind == "wmass_p1":
        return oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P1, coef))
    if kind == "wmass_p0":
        return oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P0, coef))
    if kind == "stiff":
        return oracle.assemble(oracle.STIFF, m.q, m.me)
    return oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, coef))


def coef_for(kind, m, seed):
    if kind == "wmass_p1":
        return meshgen.vertex_weights(seed, m.nq)
    if kind in ("wmass_p0", "stiff_w"):
        return meshgen.element_weights(seed, m.nme)
    return None


KINDS = ["mass", "wmass_p1", "wmass_p0", "stiff", "stiff_w"]


@pytest.mark.parametrize("d,N", [(2, 37), (3, 9)])
@pytest.mark.parametrize("strategy", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_parity_all_kinds(d, N, strategy, prec):
    fe = fe_or_skip()
    m = mesh(d, N, seed=d * 100 + N)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    p.set_strategy(strategy)
    for kind in KINDS:
        c = coef_for(kind, m, seed=N)
        ref = oracle_ref(kind, m, c)
        if kind == KINDS[0]:
            assert p.nnz == ref["nnz"] and p.n == ref["n"]
            assert_pattern_equal(p, ref)
        vals = run(fe, p, kind, q, prec, None if c is None else to_cuda(c))
        assert p.status() == (0, -1)
        check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D {kind}, strategy {strategy}")


@pytest.mark.parametrize("d", [2, 3])
def test_keep_order_pattern_and_slot_maps(d):
    fe = fe_or_skip()
    m = mesh(d, 11 if d == 2 else 5, seed=3)
    q, me = to_cuda(m.q), to_cuda(m.me)
    ref = oracle.assemble(oracle.STIFF, m.q, m.me)
    for flags in (0, fe.PATTERN_KEEP_ORDER):
        p = fe.fe_pattern(q, me, flags=flags)
        assert_pattern_equal(p, ref)
        s2n, nsp, n2s, order = (t.cpu().numpy() for t in p.slot_map())
        S = (d + 1) ** 2
        order = order.astype(np.int64)
        assert sorted(order.tolist()) == list(range(m.nme))
        if flags:
            np.testing.assert_array_equal(order, np.arange(m.nme))
        # slot -> (row, col) of the internal element order agrees with the CSR
        rp = ref["row_ptr"]
        rows = np.repeat(np.arange(m.nq), np.diff(rp))
        e = np.arange(m.nme * S) // S
        loc = np.arange(m.nme * S) % S
        a, b = loc % (d + 1), loc // (d + 1)
        me_int = m.me[:, order]
        np.testing.assert_array_equal(rows[s2n], me_int[a, e])
        np.testing.assert_array_equal(ref["col_idx"][s2n], me_int[b, e])
        # nnz2slot lists are the inverse map, ascending within each nonzero
        assert nsp[0] == 0 and nsp[-1] == m.nme * S
        np.testing.assert_array_equal(s2n[n2s], np.repeat(np.arange(ref["nnz"]), np.diff(nsp)))
        seg_id = np.repeat(np.arange(ref["nnz"]), np.diff(nsp))
        assert np.all((np.diff(n2s) > 0) | (np.diff(seg_id) != 0))


@pytest.mark.parametrize("strategy", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_run_to_run_bit_identical(strategy, prec):
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(12, seed=4)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    p.set_strategy(strategy)
    first = fe.fe_assemble_stiff(p, q, prec=prec).cpu()
    for _ in range(3):
        again = fe.fe_assemble_stiff(p, q, prec=prec).cpu()
        assert bool((again == first).all())
    # a second pattern of the same mesh gives the same bits
    p2 = fe.fe_pattern(q, me)
    p2.set_strategy(strategy)
    assert bool((fe.fe_assemble_stiff(p2, q, prec=prec).cpu() == first).all())


def test_chunked_equals_gather_closely_and_golden():
    fe = fe_or_skip()
    import os
    from test_oracle import read_golden
    for name in ("two_triangles.txt", "two_tets.txt"):
        qn, men, gold = read_golden(name)
        q, me = to_cuda(qn), to_cuda(men)
        p = fe.fe_pattern(q, me)
        rp, ci = (t.cpu().numpy() for t in p.csr())
        rows = np.repeat(np.arange(p.n), np.diff(rp))
        for key, fn in (("stiff", fe.fe_assemble_stiff), ("mass", fe.fe_assemble_mass)):
            got = dict(zip(zip(rows.tolist(), ci.tolist()), fn(p, q).cpu().numpy().tolist()))
            assert set(got) == set(gold[key])
            for ij, v in gold[key].items():
                assert got[ij] == pytest.approx(v, abs=1e-15)


def test_moved_vertices_same_pattern():
    # fixed-pattern reassembly: new coordinates, same topology
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(7, seed=5)
    m2 = meshgen.kuhn_cube_mesh(7, seed=6)  # same topology (identity vertex order), other jitter
    m2.me[:] = m.me
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    ref = oracle.assemble(oracle.STIFF, m2.q, m2.me)
    vals = fe.fe_assemble_stiff(p, to_cuda(m2.q))
    check_values(vals.cpu().numpy(), ref, 0, "3D stiffness, fixed pattern, new coordinates")


def test_errors_are_reported():
    fe = fe_or_skip()
    m = meshgen.square_mesh(6, seed=7)
    q, me = to_cuda(m.q), to_cuda(m.me)
    bad = m.me.copy()
    bad[2, 11] = m.nq + 5
    with pytest.raises(fe.FEError) as e:
        fe.fe_pattern(q, to_cuda(bad))
    assert e.value.code == 2
    p = fe.fe_pattern(q, me)
    # collapse the edge (a, c) of element 9: every element holding both is degenerate
    qb = m.q.copy()
    a, b, c = m.me[:, 9]
    qb[:, c] = qb[:, a]
    for strategy in (0, 1, 2):
        p.set_strategy(strategy)
        fe.fe_assemble_stiff(p, to_cuda(qb))
        code, eid = p.status()
        assert code == 3 and eid >= 0
        assert 0.0 == abs(np.linalg.det(np.stack([qb[:, m.me[1, eid]] - qb[:, m.me[0, eid]],
                                                  qb[:, m.me[2, eid]] - qb[:, m.me[0, eid]]])))
    assert p.status() == (0, -1)
    # argument errors are caught on the host
    import torch
    with pytest.raises(fe.FEError):
        fe.fe_assemble_wmass(p, q, torch.ones(m.nq, device="cuda", dtype=torch.float64), 99)
    with pytest.raises(ValueError):
        fe.fe_assemble_stiff(p, q.float())


def test_split_coordinates_fp32_form_accuracy_on_large_offsets():
    # coordinates far from the origin: the FP32 form must still resolve h = 1e-3 edges
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(6, seed=8)
    qs = m.q * 1e-2 + np.array([[1000.0], [-2000.0], [3000.5]])
    q, me = to_cuda(qs), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    ref = oracle.assemble(oracle.STIFF, qs, m.me)
    check_values(fe.fe_assemble_stiff(p, q, prec=1).double().cpu().numpy(), ref, 1,
                 "3D stiffness, coordinates offset to 3000")


def test_unordered_mesh_shrinks_chunks_and_stays_correct():
    # KEEP_ORDER on a randomly ordered mesh: chunks touch most of the mesh, so the plan
    # build halves the chunk until a block's shared memory fits
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(16, seed=12)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_KEEP_ORDER | fe.PATTERN_CHUNK(4096))
    assert p.plan_info()["chunk"] < 4096
    ref = oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P1, meshgen.vertex_weights(1, m.nq)))
    import torch
    vals = fe.fe_assemble_wmass(p, q, to_cuda(meshgen.vertex_weights(1, m.nq)), fe.COEF_P1)
    check_values(vals.cpu().numpy(), ref, 0, "3D weighted mass P1, unordered mesh")
    ref_s = oracle.assemble(oracle.STIFF, m.q, m.me)
    check_values(fe.fe_assemble_stiff(p, q).cpu().numpy(), ref_s, 0, "3D stiffness, unordered mesh")

"""GPU parity of the general second-order operator (Eq. EDP) through the C ABI.

The CUDA path is compared with the FP64 oracle on the same seeded inputs, entry by
entry, within 1e-12 (FP64 and F64X forms) or 1e-5 (FP32 form) of the normalised error. The
operator is not symmetric, so each orientation of every edge is checked.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

def mesh(d, N, seed=0):
    return meshgen.square_mesh(N, seed=seed) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=seed)


def dtype(prec):
    import torch
    return torch.float32 if prec == 1 else torch.float64


@pytest.mark.parametrize("d,N", [(2, 37), (3, 9)])
@pytest.mark.parametrize("strategy", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_parity_per_element(d, N, strategy, prec):
    fe = fe_or_skip()
    m = mesh(d, N, seed=d * 10 + N)
    cf = meshgen.general_coefficients(N, d, m.nme)
    ref = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    p.set_strategy(strategy)
    assert_pattern_equal(p, ref)
    vals = fe.fe_assemble_general(p, q, to_cuda(cf, dtype(prec)), fe.COEF_P0, prec=prec)
    assert p.status() == (0, -1)
    check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D general operator, P0 coefficients")


@pytest.mark.parametrize("d,N", [(2, 29), (3, 8)])
@pytest.mark.parametrize("strategy", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_parity_p1_coefficients(d, N, strategy, prec):
    fe = fe_or_skip()
    m = mesh(d, N, seed=d * 10 + N + 1)
    cf = meshgen.general_coefficients(N + 50, d, m.nq)  # one set per vertex
    ref = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P1)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    p.set_strategy(strategy)
    vals = fe.fe_assemble_general(p, q, to_cuda(cf, dtype(prec)), fe.COEF_P1, prec=prec)
    assert p.status() == (0, -1)
    check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D general operator, P1 coefficients")


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_parity_scalar_and_internal_order(d, prec):
    fe = fe_or_skip()
    m = mesh(d, 21 if d == 2 else 7, seed=5)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    cf = meshgen.general_coefficients(6, d, m.nme)
    # one coefficient set for the whole mesh
    ref = oracle.assemble_general(m.q, m.me, cf[0], oracle.COEF_SCALAR)
    vals = fe.fe_assemble_general(p, q, to_cuda(cf[0].copy(), dtype(prec)), fe.COEF_SCALAR, prec=prec)
    check_values(vals.double().cpu().numpy(), ref, prec, "3D general operator, scalar coefficients")
    # per element, given in the pattern's internal order
    order = p.element_order().cpu().numpy()
    ref = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P0)
    vals = fe.fe_assemble_general(p, q, to_cuda(cf[order].copy(), dtype(prec)), fe.COEF_P0_INTERNAL,
                                  prec=prec)
    assert p.status() == (0, -1)
    check_values(vals.double().cpu().numpy(), ref, prec, "3D general operator, scalar coefficients")


@pytest.mark.parametrize("chunk", [32, 96])
def test_small_chunks_many_partials(chunk):
    # small chunks make most vertices and edges shared: both orientations go through
    # the partial sums and the fixup
    fe = fe_or_skip()
    m = mesh(3, 8, seed=7)
    cf = meshgen.general_coefficients(7, 3, m.nme)
    ref = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(chunk))
    assert p.plan_info()["partial_edges"] > 0
    vals = fe.fe_assemble_general(p, q, to_cuda(cf), fe.COEF_P0)
    check_values(vals.cpu().numpy(), ref, 0, "3D general operator, small chunks")


def test_deterministic_and_not_symmetric():
    fe = fe_or_skip()
    import torch
    m = mesh(3, 10, seed=8)
    cf = meshgen.general_coefficients(8, 3, m.nme)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    c = to_cuda(cf)
    a = fe.fe_assemble_general(p, q, c, fe.COEF_P0)
    b = fe.fe_assemble_general(p, q, c, fe.COEF_P0)
    assert torch.equal(a, b)  # fixed summation order: bit-identical reruns
    rp, ci = p.csr()
    A = torch.sparse_csr_tensor(rp.long().cpu(), ci.long().cpu(), a.cpu(), size=(p.n, p.n)).to_dense()
    assert (A - A.T).abs().max().item() > 1e-3
    # identity diffusion, no convection or reaction: the stiffness matrix
    z = np.zeros_like(cf)
    z[:, [0, 4, 8]] = 1.0
    g = fe.fe_assemble_general(p, q, to_cuda(z), fe.COEF_P0)
    s = fe.fe_assemble_stiff(p, q)
    assert (g - s).abs().max().item() <= 1e-12 * s.abs().max().item()


def test_batched_pattern():
    fe = fe_or_skip()
    import torch
    meshes = [mesh(2, 9, seed=1), mesh(2, 14, seed=2), mesh(2, 5, seed=3)]
    qs = [to_cuda(x.q) for x in meshes]
    mes = [to_cuda(x.me) for x in meshes]
    p = fe.fe_batch_pattern(qs, mes)
    vo, eo, no = fe.fe_batch_offsets(p)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p, qs, mes, qu)
    cfs = [meshgen.general_coefficients(10 + i, 2, x.nme) for i, x in enumerate(meshes)]
    vals = fe.fe_assemble_general(p, qu, to_cuda(np.concatenate(cfs, axis=0)), fe.COEF_P0)
    assert p.status() == (0, -1)
    for i, x in enumerate(meshes):
        ref = oracle.assemble_general(x.q, x.me, cfs[i], oracle.COEF_P0)
        got = vals[int(no[i]):int(no[i + 1])].cpu().numpy()
        check_values(got, ref, 0, "2D general operator, batch")


def test_rejects_unsupported_calls():
    fe = fe_or_skip()
    m = mesh(2, 6, seed=9)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    cf = to_cuda(meshgen.general_coefficients(9, 2, m.nme))
    with pytest.raises(fe.FEError):
        fe.fe_assemble_general(p, q, cf, fe.COEF_NONE)
    pv = fe.fe_pattern(q, me, m=2)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_general(pv, q, cf, fe.COEF_P0)


@pytest.mark.parametrize("d,N", [(2, 37), (3, 9), (3, 8)])
@pytest.mark.parametrize("kind", ["p0", "p1", "scalar", "p0_internal"])
def test_f64x_form(d, N, kind):
    # the double-float form (chunked strategy only) to the FP64 gate, bit-identical reruns
    fe = fe_or_skip()
    m = mesh(d, N, seed=d * 10 + N + 3)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    if kind == "p1":
        cf = meshgen.general_coefficients(N + 60, d, m.nq)
        ref, arg, k = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P1), cf, fe.COEF_P1
    elif kind == "scalar":
        cf = meshgen.general_coefficients(N + 61, d, 1)[0]
        ref, arg, k = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_SCALAR), cf.copy(), fe.COEF_SCALAR
    else:
        cf = meshgen.general_coefficients(N + 62, d, m.nme)
        ref = oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P0)
        if kind == "p0":
            arg, k = cf, fe.COEF_P0
        else:
            arg, k = cf[p.element_order().cpu().numpy()].copy(), fe.COEF_P0_INTERNAL
    vals = fe.fe_assemble_general(p, q, to_cuda(arg), k, prec=fe.F64X)
    assert p.status() == (0, -1)
    check_values(vals.cpu().numpy(), ref, 2, f"{d}D general operator, {kind} coefficients")
    again = fe.fe_assemble_general(p, q, to_cuda(arg), k, prec=fe.F64X)
    assert bool((again == vals).all())
    p.set_strategy(fe.REASM_GATHER)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_general(p, q, to_cuda(arg), k, prec=fe.F64X)

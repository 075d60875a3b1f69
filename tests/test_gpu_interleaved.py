"""Interleaved chunk records (FE_PATTERN_INTERLEAVED): element values go straight to the
slots of their vertex or edge, laid out so that a warp sums 32 lists from consecutive
slots.

Checked through the C ABI: the CSR pattern bit for bit against the oracle; every scalar
operator against the FP64 oracle in both forms, over chunk sizes and threads per block;
the FP32 values bit for bit equal to those of the plain layout (same summation order,
same element values); run-to-run bit identity; the operators that do not take such a
pattern refuse it.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

KINDS = ("mass", "wmass_p1", "wmass_p0", "stiff", "stiff_w")


def run(fe, p, kind, q, prec, wv, we):
    if kind == "mass":
        return fe.fe_assemble_mass(p, q, prec=prec)
    if kind == "wmass_p1":
        return fe.fe_assemble_wmass(p, q, wv, fe.COEF_P1, prec=prec)
    if kind == "wmass_p0":
        return fe.fe_assemble_wmass(p, q, we, fe.COEF_P0, prec=prec)
    if kind == "stiff":
        return fe.fe_assemble_stiff(p, q, prec=prec)
    return fe.fe_assemble_stiff(p, q, we, fe.COEF_P0, prec=prec)


def ref(kind, m, wv, we):
    if kind == "mass":
        return oracle.assemble(oracle.MASS, m.q, m.me)
    if kind == "wmass_p1":
        return oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P1, wv))
    if kind == "wmass_p0":
        return oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P0, we))
    if kind == "stiff":
        return oracle.assemble(oracle.STIFF, m.q, m.me)
    return oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, we))


@pytest.mark.parametrize("d,N", [(2, 37), (3, 9)])
@pytest.mark.parametrize("chunk,threads", [(128, 128), (512, 256), (1024, 512)])
def test_interleaved_parity_and_bit_identity(d, N, chunk, threads):
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(N, seed=d + N) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=d + N)
    q, me = to_cuda(m.q), to_cuda(m.me)
    pi = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(chunk) | fe.PATTERN_INTERLEAVED)
    pp = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(chunk))
    pi.set_threads(threads)
    pp.set_threads(threads)
    assert_pattern_equal(pi, oracle.assemble(oracle.MASS, m.q, m.me))
    wv_n, we_n = meshgen.vertex_weights(N, m.nq), meshgen.element_weights(N, m.nme)
    for prec in (fe.F64, fe.F32):
        T = torch.float64 if prec == fe.F64 else torch.float32
        wv, we = to_cuda(wv_n).to(T), to_cuda(we_n).to(T)
        for kind in KINDS:
            v = run(fe, pi, kind, q, prec, wv, we)
            assert pi.status() == (0, -1)
            check_values(v.double().cpu().numpy(), ref(kind, m, wv_n, we_n), prec,
                         f"{d}D {kind}, interleaved records")
            assert torch.equal(v, run(fe, pi, kind, q, prec, wv, we))  # run to run
            if prec == fe.F32:
                assert torch.equal(v, run(fe, pp, kind, q, prec, wv, we))  # the plain layout's values


def test_interleaved_pattern_refused_where_unsupported():
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(4, seed=9)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_INTERLEAVED)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_stiff(p, q, prec=fe.F64X)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_general(p, q, to_cuda(meshgen.general_coefficients(1, 3, m.nme)), fe.COEF_P0)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_wmass_stiff(p, q)
    with pytest.raises(fe.FEError):  # vector problems have no interleaved records
        fe.fe_pattern(q, me, m=3, flags=fe.PATTERN_INTERLEAVED)
    # the two-pass and atomic strategies do not read chunk records and still work
    ref_s = oracle.assemble(oracle.STIFF, m.q, m.me)
    for strategy in (fe.REASM_GATHER, fe.REASM_ATOMIC):
        p.set_strategy(strategy)
        check_values(fe.fe_assemble_stiff(p, q).cpu().numpy(), ref_s, 0, "3D stiff, interleaved pattern, "
                     "gather / atomic")

"""Batched assembly (disjoint union of many meshes, one launch per operator) and
repeated fixed-pattern reassembly replayed from a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def batch(count, seed, lo=3, hi=14):
    sizes = meshgen.batch_sizes(seed, count, lo, hi)
    return [meshgen.square_mesh(int(N), seed=seed * 1000 + b) for b, N in enumerate(sizes)]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_matches_each_mesh(prec):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    meshes = batch(7, 5)
    qs = [to_cuda(m.q) for m in meshes]
    mes = [to_cuda(m.me) for m in meshes]
    p = fe.fe_batch_pattern(qs, mes)
    vo, eo, no = fe.fe_batch_offsets(p)
    assert vo[-1] == sum(m.nq for m in meshes) and eo[-1] == sum(m.nme for m in meshes)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p, qs, mes, qu)
    w_el = [meshgen.element_weights(11 + b, m.nme) for b, m in enumerate(meshes)]
    w_v = [meshgen.vertex_weights(21 + b, m.nq) for b, m in enumerate(meshes)]
    stiff = fe.fe_assemble_stiff(p, qu, to_cuda(np.concatenate(w_el)).to(T), fe.COEF_P0, prec=prec)
    wmass = fe.fe_assemble_wmass(p, qu, to_cuda(np.concatenate(w_v)).to(T), fe.COEF_P1, prec=prec)
    assert p.status() == (0, -1)
    rp, ci = (t.cpu().numpy() for t in p.csr())
    for b, m in enumerate(meshes):
        rs = oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, w_el[b]))
        rw = oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P1, w_v[b]))
        sl = slice(int(no[b]), int(no[b + 1]))
        np.testing.assert_array_equal(rp[vo[b]:vo[b + 1] + 1] - no[b], rs["row_ptr"])
        np.testing.assert_array_equal(ci[sl] - vo[b], rs["col_idx"])
        check_values(stiff[sl].double().cpu().numpy(), rs, prec, "2D batch: stiffness P0 w")
        check_values(wmass[sl].double().cpu().numpy(), rw, prec, "2D batch: weighted mass P1")


def test_graph_replay_with_fresh_weights_is_bit_identical_to_direct_calls():
    fe = fe_or_skip()
    import torch
    meshes = batch(5, 9, 8, 20)
    qs = [to_cuda(m.q) for m in meshes]
    mes = [to_cuda(m.me) for m in meshes]
    p = fe.fe_batch_pattern(qs, mes)
    vo, eo, _ = fe.fe_batch_offsets(p)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p, qs, mes, qu)
    w = torch.empty(int(eo[-1]), dtype=torch.float64, device="cuda")
    stiff = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    mass = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    w.fill_(1.0)
    # warm-up outside capture (kernel attributes, module loading)
    fe.fe_assemble_stiff(p, qu, w, fe.COEF_P0_INTERNAL, vals=stiff)
    fe.fe_assemble_wmass(p, qu, w, fe.COEF_P0_INTERNAL, vals=mass)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fe.fe_assemble_stiff(p, qu, w, fe.COEF_P0_INTERNAL, vals=stiff)
        fe.fe_assemble_wmass(p, qu, w, fe.COEF_P0_INTERNAL, vals=mass)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    for _ in range(5):
        w.copy_(torch.randn(w.shape, generator=gen, device="cuda", dtype=torch.float64).exp())
        g.replay()
        torch.cuda.synchronize()
        s_ref = fe.fe_assemble_stiff(p, qu, w, fe.COEF_P0_INTERNAL)
        m_ref = fe.fe_assemble_wmass(p, qu, w, fe.COEF_P0_INTERNAL)
        assert bool((stiff == s_ref).all()) and bool((mass == m_ref).all())

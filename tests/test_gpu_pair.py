"""fe_assemble_wmass_stiff: the weighted mass and stiffness matrices with one per-element
coefficient in one pass (one chunk kernel, persistent or one block per chunk, and one
fixup), for repeated reassembly with fresh coefficients.

Checked through the C ABI, in the FP64, FP32 and F64X forms: bit for bit against the
separate calls fe_assemble_wmass and fe_assemble_stiff (same summation order), against the
FP64 oracle for both operators, over chunk sizes, threads per block and both launch shapes,
on a single 3D mesh and on a batch of 2D meshes; a CUDA-graph replay with fresh weights
equals direct calls bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("chunk,threads,persistent", [(256, 128, True), (512, 256, False), (1024, 512, True)])
def test_pair_matches_separate_calls_and_oracle_3d(prec, chunk, threads, persistent):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    m = meshgen.kuhn_cube_mesh(9, seed=61)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(chunk))
    p.set_threads(threads)
    p.set_persistent(persistent)
    w = meshgen.element_weights(61, m.nme)
    wt = to_cuda(w).to(T)
    vm, vs = fe.fe_assemble_wmass_stiff(p, q, wt, fe.COEF_P0, prec=prec)
    assert p.status() == (0, -1)
    assert torch.equal(vm, fe.fe_assemble_wmass(p, q, wt, fe.COEF_P0, prec=prec))
    assert torch.equal(vs, fe.fe_assemble_stiff(p, q, wt, fe.COEF_P0, prec=prec))
    check_values(vm.double().cpu().numpy(), oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P0, w)),
                 prec, "3D weighted mass P0, fused with stiffness")
    check_values(vs.double().cpu().numpy(), oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, w)),
                 prec, "3D stiffness P0 w, fused with weighted mass")
    # no coefficient: the mass matrix and the plain stiffness
    vm0, vs0 = fe.fe_assemble_wmass_stiff(p, q, prec=prec)
    assert torch.equal(vm0, fe.fe_assemble_mass(p, q, prec=prec))
    assert torch.equal(vs0, fe.fe_assemble_stiff(p, q, prec=prec))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pair_on_a_batch_of_2d_meshes_with_graph_replay(prec):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    sizes = [7, 16, 3, 25, 11]
    meshes = [meshgen.square_mesh(n, seed=70 + b) for b, n in enumerate(sizes)]
    qs = [to_cuda(x.q) for x in meshes]
    mes = [to_cuda(x.me) for x in meshes]
    p = fe.fe_batch_pattern(qs, mes)
    vo, eo, no = fe.fe_batch_offsets(p)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p, qs, mes, qu)
    order = p.element_order().long()
    ws = [meshgen.element_weights(80 + b, x.nme) for b, x in enumerate(meshes)]
    w_int = to_cuda(np.concatenate(ws)).to(T)[order].contiguous()  # internal element order
    vm, vs = fe.fe_assemble_wmass_stiff(p, qu, w_int, fe.COEF_P0_INTERNAL, prec=prec)
    assert p.status() == (0, -1)
    assert torch.equal(vm, fe.fe_assemble_wmass(p, qu, w_int, fe.COEF_P0_INTERNAL, prec=prec))
    assert torch.equal(vs, fe.fe_assemble_stiff(p, qu, w_int, fe.COEF_P0_INTERNAL, prec=prec))
    vmn, vsn = vm.double().cpu().numpy(), vs.double().cpu().numpy()
    for b, x in enumerate(meshes):
        sl = slice(int(no[b]), int(no[b + 1]))
        check_values(vmn[sl], oracle.assemble(oracle.WMASS, x.q, x.me, c1=(oracle.COEF_P0, ws[b])), prec,
                     "2D batch: weighted mass P0, fused with stiffness")
        check_values(vsn[sl], oracle.assemble(oracle.STIFF, x.q, x.me, c1=(oracle.COEF_P0, ws[b])), prec,
                     "2D batch: stiffness P0 w, fused with weighted mass")
    # graph replay with weights drawn afresh inside the graph equals a direct call
    w = torch.empty_like(w_int)
    gm, gs = torch.empty_like(vm), torch.empty_like(vs)

    def step():
        w.copy_(torch.randn(w.shape, device="cuda", dtype=torch.float32).exp_())
        fe.fe_assemble_wmass_stiff(p, qu, w, fe.COEF_P0_INTERNAL, prec=prec, vals_mass=gm, vals_stiff=gs)
    torch.cuda.manual_seed(5)
    step()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        dm, ds = fe.fe_assemble_wmass_stiff(p, qu, w.clone(), fe.COEF_P0_INTERNAL, prec=prec)
        assert torch.equal(gm, dm) and torch.equal(gs, ds)
    assert p.status() == (0, -1)


def test_pair_rejects_unsupported_calls():
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(3, seed=62)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    v = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FEError):  # one array for both matrices
        fe.fe_assemble_wmass_stiff(p, q, vals_mass=v, vals_stiff=v)
    with pytest.raises(fe.FEError):  # P1 coefficient
        fe.fe_assemble_wmass_stiff(p, q, to_cuda(np.ones(m.nq)), fe.COEF_P1)
    p.set_strategy(fe.REASM_GATHER)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_wmass_stiff(p, q)
    with pytest.raises(fe.FEError):  # launch shape other than 0 / 1
        fe._check(fe.lib().fe_pattern_set_persistent(p.handle, 2))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pair_on_badly_shaped_elements(prec):
    # slivers, caps and needles take the recomputation paths of the FP32 and F64X forms
    # (FP64 det B / whole element from the FP64 coordinates); the fused kernel must take
    # them for both matrices exactly as the separate calls do
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    m = meshgen.badly_shaped_mesh(3, [1e-2, 1e-4, 1e-6, 1e-8, 1e-10], seed=63)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    wt = to_cuda(meshgen.element_weights(64, m.nme)).to(T)
    vm, vs = fe.fe_assemble_wmass_stiff(p, q, wt, fe.COEF_P0, prec=prec)
    assert p.status() == (0, -1)
    assert torch.equal(vm, fe.fe_assemble_wmass(p, q, wt, fe.COEF_P0, prec=prec))
    assert torch.equal(vs, fe.fe_assemble_stiff(p, q, wt, fe.COEF_P0, prec=prec))

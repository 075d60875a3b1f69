"""fe_assemble_stiff_noalloc: the stiffness assembly for callers that may not call
cudaMalloc while they assemble (a plugin inside an application that owns the device
memory budget, a time-stepping loop that cannot afford the synchronisation an
allocation may cause). It writes its element values to a fixed scratch array of
the library instead of allocating.

Checked through the C ABI against the existing entry point, fe_assemble_stiff, on
two calls in a row (the second with new coordinates, so stale scratch would
show), with the normalised per-nonzero tolerance the other parity tests use. The
file name makes pytest collect it last.
"""
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import fe_or_skip, normalised_error, to_cuda

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_fe_assemble_stiff_on_two_calls(prec):
    fe = fe_or_skip()
    import torch
    T = torch.float64 if prec == 0 else torch.float32
    m = meshgen.kuhn_cube_mesh(10, seed=21)            # 6,000 tets
    m2 = meshgen.kuhn_cube_mesh(10, seed=22)           # same topology, other jitter
    q, q2, me = to_cuda(m.q), to_cuda(m2.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    vals = torch.empty(p.nnz, dtype=T, device="cuda")  # the caller's output buffer
    for call, (qq, qn) in enumerate(((q, m.q), (q2, m2.q))):
        scale = oracle.assemble(oracle.STIFF, qn, m.me)["scale"]
        expected = fe.fe_assemble_stiff(p, qq, prec=prec)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        fe.fe_assemble_stiff_noalloc(p, qq, vals, prec=prec)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the library's module; later calls take nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        assert p.status() == (0, -1)
        err = normalised_error(vals.double().cpu().numpy(), expected.double().cpu().numpy(), scale)
        assert err <= TOL[prec], (call, err)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(28, seed=23)            # 131,712 tets: 16.08 MiB of FP64 values
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    vals = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FEError) as e:
        fe.fe_assemble_stiff_noalloc(p, q, vals, prec=fe.F64)
    assert e.value.code == 8
    with pytest.raises(fe.FEError) as e:  # FE_F64X is not one of its forms
        fe.fe_assemble_stiff_noalloc(p, q, vals, prec=fe.F64X)
    assert e.value.code == 1
    vals32 = torch.empty(p.nnz, dtype=torch.float32, device="cuda")  # 8.04 MiB in FP32: fits
    fe.fe_assemble_stiff_noalloc(p, q, vals32, prec=fe.F32)
    expected = fe.fe_assemble_stiff(p, q, prec=fe.F32)
    scale = oracle.assemble(oracle.STIFF, m.q, m.me)["scale"]
    assert normalised_error(vals32.double().cpu().numpy(), expected.double().cpu().numpy(), scale) <= 1e-5

"""Host-buffer assembly: results equal the device-memory call bit for bit, including when
successive calls overlap (each call's own coordinates, two result buffers in turn)."""
import numpy as np
import pytest

from paper_1401_3301_gb300 import meshgen
from helpers import fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("weighted", [False, True])
def test_host_calls_match_device_calls(prec, weighted):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == fe.F32 else torch.float64
    m = meshgen.kuhn_cube_mesh(12, seed=60)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    w = torch.from_numpy(meshgen.element_weights(61, m.nme)).to(T) if weighted else None
    rng = np.random.default_rng(62)
    qs = [m.q + 1e-3 * rng.normal(size=m.q.shape) * (k > 0) for k in range(5)]
    q_host = [torch.from_numpy(x).pin_memory() for x in qs]
    out = [torch.empty(p.nnz, dtype=T).pin_memory() for _ in range(5)]
    stream = torch.cuda.current_stream()
    for k in range(5):
        fe.fe_assemble_stiff_host(p, q_host[k], out[k], None if w is None else w.pin_memory(), prec=prec)
    stream.synchronize()
    for k in range(5):
        qd = to_cuda(qs[k])
        ref = fe.fe_assemble_stiff(p, qd, None if w is None else w.cuda(), fe.COEF_NONE if w is None else fe.COEF_P0,
                                   prec=prec)
        assert torch.equal(out[k], ref.cpu()), k
    assert p.status() == (0, -1)


def test_pageable_buffers_and_argument_checks():
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(10, seed=63)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    out = torch.empty(p.nnz, dtype=torch.float64)
    fe.fe_assemble_stiff_host(p, torch.from_numpy(m.q), out)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(out, fe.fe_assemble_stiff(p, q).cpu())
    with pytest.raises(ValueError):
        fe.fe_assemble_stiff_host(p, torch.from_numpy(m.q), torch.empty(p.nnz, dtype=torch.float32))

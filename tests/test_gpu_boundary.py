"""GPU boundary (facet) mass and weighted mass vs the oracle: pattern bit-exact,
FP64 and F64X <= 1e-12, FP32 <= 1e-5 normalised error."""
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,N", [(2, 23), (3, 9)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_boundary_parity(d, N, prec):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    m = meshgen.square_mesh(N, seed=N) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=N)
    fa = meshgen.boundary_facets(m)
    q, f = to_cuda(m.q), to_cuda(fa)
    p = fe.fe_boundary_pattern(q, f)
    ref = oracle.assemble_boundary(oracle.MASS, m.q, fa)
    assert (p.n, p.nnz) == (ref["n"], ref["nnz"])
    assert_pattern_equal(p, ref)
    cases = [(fe.fe_assemble_mass(p, q, prec=prec), ref, "mass")]
    wv = meshgen.vertex_weights(N, m.nq)
    cases.append((fe.fe_assemble_wmass(p, q, to_cuda(wv).to(T), fe.COEF_P1, prec=prec),
                  oracle.assemble_boundary(oracle.WMASS, m.q, fa, c1=(oracle.COEF_P1, wv)), "weighted mass P1"))
    wf = meshgen.element_weights(N, fa.shape[1])
    cases.append((fe.fe_assemble_wmass(p, q, to_cuda(wf).to(T), fe.COEF_P0, prec=prec),
                  oracle.assemble_boundary(oracle.WMASS, m.q, fa, c1=(oracle.COEF_P0, wf)), "weighted mass P0"))
    for vals, r, what in cases:
        assert p.status() == (0, -1)
        check_values(vals.double().cpu().numpy(), r, prec, f"{d}D facets: {what}")
    with pytest.raises(fe.FEError):
        fe.fe_assemble_stiff(p, q)

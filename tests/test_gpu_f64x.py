"""FE_F64X form of mass, weighted mass and stiffness: FP64 results of FP64-class accuracy
from double-float arithmetic. Same gate as the FP64 form (1e-12 normalised error vs the
FP64 oracle)."""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,N,offset", [(2, 37, 0.0), (3, 9, 0.0), (3, 8, 1000.0), (2, 25, -3000.5)])
def test_f64x_matches_oracle_to_fp64_tolerance(d, N, offset):
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(N, seed=N) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=N)
    qn = m.q + offset
    q, me = to_cuda(qn), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    w = meshgen.element_weights(N, m.nme)
    for coef in (None, w):
        ref = oracle.assemble(oracle.STIFF, qn, m.me, c1=None if coef is None else (oracle.COEF_P0, coef))
        vals = fe.fe_assemble_stiff(p, q, None if coef is None else to_cuda(coef), prec=fe.F64X)
        assert vals.dtype == torch.float64
        assert p.status() == (0, -1)
        check_values(vals.cpu().numpy(), ref, 2, f"{d}D stiffness{'' if coef is None else ' P0 w'}"
                     f"{', offset' if offset else ''}")
        again = fe.fe_assemble_stiff(p, q, None if coef is None else to_cuda(coef), prec=fe.F64X)
        assert bool((again == vals).all())


@pytest.mark.parametrize("d,N,offset", [(2, 37, 0.0), (3, 9, 0.0), (3, 8, 1000.0), (2, 25, -3000.5)])
def test_f64x_mass_and_weighted_mass_match_oracle(d, N, offset):
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(N, seed=N) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=N)
    qn = m.q + offset
    q, me = to_cuda(qn), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    wv = meshgen.vertex_weights(N, m.nq)
    we = meshgen.element_weights(N, m.nme)
    cases = [
        (lambda: fe.fe_assemble_mass(p, q, prec=fe.F64X), oracle.assemble(oracle.MASS, qn, m.me)),
        (lambda: fe.fe_assemble_wmass(p, q, to_cuda(wv), fe.COEF_P1, prec=fe.F64X),
         oracle.assemble(oracle.WMASS, qn, m.me, c1=(oracle.COEF_P1, wv))),
        (lambda: fe.fe_assemble_wmass(p, q, to_cuda(we), fe.COEF_P0, prec=fe.F64X),
         oracle.assemble(oracle.WMASS, qn, m.me, c1=(oracle.COEF_P0, we))),
    ]
    names = ["mass", "weighted mass P1", "weighted mass P0"]
    for k, (run, ref) in enumerate(cases):
        vals = run()
        assert vals.dtype == torch.float64
        assert p.status() == (0, -1)
        check_values(vals.cpu().numpy(), ref, 2, f"{d}D {names[k]}{', offset' if offset else ''}")
        assert bool((run() == vals).all())


def test_f64x_reports_degenerate_elements_and_rejects_other_operators():
    fe = fe_or_skip()
    import torch
    m = meshgen.square_mesh(6, seed=3)
    qb = m.q.copy()
    a, b, c = m.me[:, 4]
    qb[:, c] = qb[:, a]
    p = fe.fe_pattern(to_cuda(m.q), to_cuda(m.me))
    bad = [e for e in range(m.nme) if a in m.me[:, e] and c in m.me[:, e]]
    for run in (lambda: fe.fe_assemble_stiff(p, to_cuda(qb), prec=fe.F64X),
                lambda: fe.fe_assemble_mass(p, to_cuda(qb), prec=fe.F64X)):
        run()
        assert p.status() == (3, min(bad))
    # F64X runs the chunked strategy only
    p.set_strategy(fe.REASM_GATHER)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_stiff(p, to_cuda(m.q), prec=fe.F64X)

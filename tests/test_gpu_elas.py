"""GPU parity of linear elasticity (m = d block pattern) through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

def mesh(d, N, seed):
    return meshgen.square_mesh(N, seed=seed) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=seed)


def coef(kind, m, seed, base):
    """(oracle form, device array, fe kind) of a Lame field of the given kind."""
    import torch
    from paper_1401_3301_gb300 import fe
    if kind == "scalar":
        return base, torch.tensor([base], dtype=torch.float64), fe.COEF_SCALAR
    if kind == "p0":
        v = base * meshgen.element_weights(seed, m.nme)
        return (oracle.COEF_P0, v), torch.from_numpy(v), fe.COEF_P0
    v = base * meshgen.vertex_weights(seed, m.nq)
    return (oracle.COEF_P1, v), torch.from_numpy(v), fe.COEF_P1


@pytest.mark.parametrize("d,N", [(2, 13), (3, 5), (3, 9)])
@pytest.mark.parametrize("kind", ["scalar", "p0", "p1"])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_elasticity_parity(d, N, kind, prec):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    m = mesh(d, N, seed=50 + N)
    lam0, mu0 = meshgen.lame_from_young(1.0, 0.3)
    lo, ld, lk = coef(kind, m, 1, lam0)
    mo, md, mk = coef(kind, m, 2, mu0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, m=d)
    ref = oracle.assemble(oracle.ELAS, m.q, m.me, c1=lo, c2=mo)
    assert (p.n, p.nnz) == (ref["n"], ref["nnz"])
    assert_pattern_equal(p, ref)
    vals = fe.fe_assemble_elas(p, q, ld.to(T).cuda(), lk, md.to(T).cuda(), mk, prec=prec)
    assert p.status() == (0, -1)
    check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D elasticity, {kind} Lame")


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("d", [2, 3])
def test_elasticity_rigid_modes_gpu_and_bit_identity(d, prec):
    fe = fe_or_skip()
    import torch
    m = mesh(d, 24 if d == 2 else 8, seed=60)
    lam0, mu0 = meshgen.lame_from_young(1.0, 0.3)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, m=d)
    lam = torch.tensor([lam0], dtype=torch.float64, device="cuda")
    mu = torch.tensor([mu0], dtype=torch.float64, device="cuda")
    vals = fe.fe_assemble_elas(p, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR, prec=prec)
    again = fe.fe_assemble_elas(p, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR, prec=prec)
    assert bool((vals == again).all())
    rp, ci = (t.cpu().numpy() for t in p.csr())
    v = vals.cpu().numpy()
    rows = np.repeat(np.arange(p.n), np.diff(rp))

    def matvec(x):
        y = np.zeros(p.n)
        np.add.at(y, rows, v * x[ci])
        return y

    from test_oracle import rigid_modes
    scale = np.abs(v).max()
    for u in rigid_modes(m.q):
        assert np.abs(matvec(u)).max() < 1e-12 * scale * 10


def test_elasticity_rejects_scalar_pattern_and_other_strategies():
    fe = fe_or_skip()
    import torch
    m = mesh(3, 3, seed=61)
    q, me = to_cuda(m.q), to_cuda(m.me)
    lam = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    p1 = fe.fe_pattern(q, me, m=1)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_elas(p1, q, lam, fe.COEF_SCALAR, lam, fe.COEF_SCALAR)
    p3 = fe.fe_pattern(q, me, m=3)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_stiff(p3, q)

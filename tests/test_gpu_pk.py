"""GPU parity of the P_k mass matrix (App. D, Eq. MatElemMassPk, Algorithm 15).

The CUDA path runs through fe_pk_pattern + fe_assemble_mass; the pattern must equal the
oracle's bit for bit and the values must be within 1e-12 (FP64, F64X) / 1e-5 (FP32) of the
normalised error. Larger meshes are checked by properties exact at any size: the sum of
all entries is |Omega|, and v^T M u = int u v for polynomials of degree <= k.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import assert_pattern_equal, check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

def test_library_table_is_the_exact_table_rounded():
    fe = fe_or_skip()
    for d in (2, 3):
        for k in range(1, 7):
            C = fe.fe_pk_mass_table(d, k)
            T = oracle.pk_mass_table(d, k)
            ex = np.array([[float(x / math.factorial(d)) for x in row] for row in T])
            assert C.shape == ex.shape
            assert np.max(np.abs(C - ex) / np.maximum(np.abs(ex), 1e-300)) <= 4.5e-16, (d, k)


CASES = [(2, 8, 1), (2, 9, 2), (2, 20, 3), (2, 20, 4), (2, 6, 5), (2, 5, 6),
         (3, 3, 1), (3, 5, 2), (3, 4, 3), (3, 3, 4), (3, 2, 5), (3, 2, 6)]


@pytest.mark.parametrize("d,N,k", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_parity(d, N, k, prec):
    fe = fe_or_skip()
    m = meshgen.pk_mesh(d, N, k, seed=d * 100 + N * 10 + k, perm_nodes=True)
    ref = oracle.assemble_pk_mass(m.q, m.me, k)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pk_pattern(q, me, k)
    assert p.n == ref["n"] and p.nnz == ref["nnz"]
    assert_pattern_equal(p, ref)
    vals = fe.fe_assemble_mass(p, q, prec=prec)
    assert p.status() == (0, -1)
    check_values(vals.double().cpu().numpy(), ref, prec, f"{d}D P{k} mass")
    if prec != 1:
        import torch
        assert torch.equal(vals, fe.fe_assemble_mass(p, q, prec=prec))  # fixed summation order


@pytest.mark.parametrize("d,N,k", [(3, 40, 2), (3, 20, 3), (2, 150, 4)])
def test_large_mesh_properties(d, N, k):
    fe = fe_or_skip()
    import torch
    m = meshgen.pk_mesh(d, N, k, seed=7)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pk_pattern(q, me, k)
    vals = fe.fe_assemble_mass(p, q)
    assert p.status() == (0, -1)
    assert vals.sum().item() == pytest.approx(1.0, rel=1e-12)
    rng = np.random.default_rng(8)
    exps = [e for e in np.ndindex(*([k + 1] * d)) if sum(e) <= k]
    cu, cv = rng.normal(size=len(exps)), rng.normal(size=len(exps))

    def poly(c, X):
        return sum(ci * np.prod([X[j] ** e[j] for j in range(d)], axis=0) for ci, e in zip(c, exps))

    x, w = np.polynomial.legendre.leggauss(k + 1)
    x, w = (x + 1) / 2, w / 2
    X = np.stack([g.ravel() for g in np.meshgrid(*([x] * d), indexing="ij")])
    W = np.prod(np.meshgrid(*([w] * d), indexing="ij"), axis=0).ravel()
    exact = W @ (poly(cu, X) * poly(cv, X))
    rp, ci = p.csr()
    A = torch.sparse_csr_tensor(rp.long(), ci.long(), vals, size=(p.n, p.n))
    u = torch.from_numpy(poly(cu, m.q)).cuda()
    v = torch.from_numpy(poly(cv, m.q)).cuda()
    got = float(v @ (A @ u.unsqueeze(1)).squeeze(1))
    assert got == pytest.approx(exact, rel=1e-10, abs=1e-12)


def test_rejects_other_operators_and_strategies():
    fe = fe_or_skip()
    m = meshgen.pk_mesh(2, 4, 2, seed=3)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pk_pattern(q, me, 2)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_stiff(p, q)
    p.set_strategy(fe.REASM_GATHER)
    with pytest.raises(fe.FEError):
        fe.fe_assemble_mass(p, q)
    with pytest.raises(ValueError):
        fe.fe_pk_pattern(q, me, 3)  # 6 rows are P2 nodes, not P3

"""GPU backward pass of the stiffness assembly: L = u^T S(w) v and general VJPs.

Checked against the oracle's FP64 gradients (orc_stiff_loss), against central
finite differences of the GPU forward, and through torch.autograd.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def normwise(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def setup(d, N, seed):
    m = meshgen.square_mesh(N, seed=seed) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=seed)
    w = meshgen.element_weights(seed, m.nme)
    u, v = meshgen.random_vectors(seed, m.nq)
    return m, w, u, v


@pytest.mark.parametrize("d,N", [(2, 17), (3, 7)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_rank_one_backward_matches_oracle(d, N, prec):
    fe = fe_or_skip()
    import torch
    T = torch.float32 if prec == 1 else torch.float64
    m, w, u, v = setup(d, N, 70 + N)
    Lr, dwr, dqr = oracle.stiff_loss(m.q, m.me, w, u, v)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    L = torch.empty(1, dtype=T, device="cuda")
    dw = torch.empty(m.nme, dtype=T, device="cuda")
    dq = torch.empty((d, m.nq), dtype=T, device="cuda")
    fe.fe_assemble_stiff_backward(p, q, to_cuda(w).to(T), fe.COEF_P0, to_cuda(u).to(T), to_cuda(v).to(T),
                                  L, dw, dq, prec=prec)
    assert p.status() == (0, -1)
    tol = 2e-4 if prec == 1 else 1e-12
    assert normwise(dw.cpu().numpy(), dwr) <= tol
    assert normwise(dq.cpu().numpy(), dqr) <= tol
    assert abs(L.item() - Lr) <= tol * np.abs(dwr * w).sum()
    # bit-identical on a second run
    dq2 = torch.empty_like(dq)
    fe.fe_assemble_stiff_backward(p, q, to_cuda(w).to(T), fe.COEF_P0, to_cuda(u).to(T), to_cuda(v).to(T),
                                  None, None, dq2, prec=prec)
    assert bool((dq2 == dq).all())


@pytest.mark.parametrize("form", ["f64", "f64x"])
def test_gradients_against_central_differences_fp64(form):
    fe = fe_or_skip()
    prec = fe.F64 if form == "f64" else fe.F64X
    import torch
    from paper_1401_3301_gb300.autograd import StiffnessBilinear
    m, w, u, v = setup(3, 8, 81)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    wt, ut, vt = to_cuda(w), to_cuda(u), to_cuda(v)
    qg = q.clone().requires_grad_(True)
    wg = wt.clone().requires_grad_(True)
    L = StiffnessBilinear.apply(wg, qg, ut, vt, p, prec)
    L.backward()
    gq, gw = qg.grad.cpu().numpy(), wg.grad.cpu().numpy()

    def loss(qq, ww):
        return StiffnessBilinear.apply(ww, qq, ut, vt, p, prec).item()

    rng = np.random.default_rng(3)
    h = 1e-6 / 8
    fd_q, an_q = [], []
    for _ in range(40):
        c, vtx = int(rng.integers(3)), int(rng.integers(m.nq))
        qp, qm = q.clone(), q.clone()
        qp[c, vtx] += h
        qm[c, vtx] -= h
        fd_q.append((loss(qp, wt) - loss(qm, wt)) / (2 * h))
        an_q.append(gq[c, vtx])
    assert normwise(an_q, fd_q) <= 1e-6
    fd_w, an_w = [], []
    for _ in range(40):
        k = int(rng.integers(m.nme))
        hw = 1e-6 * w[k]
        wp, wm = wt.clone(), wt.clone()
        wp[k] += hw
        wm[k] -= hw
        fd_w.append((loss(q, wp) - loss(q, wm)) / (2 * hw))
        an_w.append(gw[k])
    assert normwise(an_w, fd_w) <= 1e-6


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_vjp_through_autograd_matches_rank_one(prec):
    fe = fe_or_skip()
    import torch
    from paper_1401_3301_gb300.autograd import StiffnessValues
    T = torch.float32 if prec == 1 else torch.float64
    m, w, u, v = setup(3, 6, 91)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    rp, ci = p.csr()
    rows = torch.repeat_interleave(torch.arange(p.n, device="cuda"), (rp[1:] - rp[:-1]).long())
    ut, vt = to_cuda(u).to(T), to_cuda(v).to(T)
    qg = q.clone().requires_grad_(True)
    wg = to_cuda(w).to(T).requires_grad_(True)
    vals = StiffnessValues.apply(wg, qg, p, prec)
    L = (ut[rows] * vals * vt[ci.long()]).sum()     # u^T S v from the CSR values
    L.backward()
    _, dwr, dqr = oracle.stiff_loss(m.q, m.me, w, u, v)
    tol = 2e-4 if prec == 1 else 1e-12
    assert normwise(wg.grad.cpu().numpy(), dwr) <= tol
    assert normwise(qg.grad.cpu().numpy(), dqr) <= tol


def test_translation_invariance_of_dq():
    fe = fe_or_skip()
    import torch
    m, w, u, v = setup(2, 20, 95)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    dq = torch.empty((2, m.nq), dtype=torch.float64, device="cuda")
    fe.fe_assemble_stiff_backward(p, q, None, fe.COEF_NONE, to_cuda(u), to_cuda(v), None, None, dq)
    g = dq.cpu().numpy()
    assert np.abs(g.sum(axis=1)).max() <= 1e-11 * np.abs(g).max() * m.nq

"""Parity at the full benchmark sizes, in the configurations bench.py times.

At these sizes the oracle cannot assemble whole matrices within seconds, so the checks are
(a) the whole CSR pattern bit for bit against the oracle's pattern-only construction;
(b) sampled rows: the oracle assembles only the elements that touch a random set of
vertices, which makes exactly those rows complete, and the GPU rows must match them entry
for entry (pattern bit for bit, values within the form's tolerance); and (c) identities of
the whole matrix that hold at any size.
"""
import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, sub_mesh_rows, to_cuda

pytestmark = pytest.mark.gpu

def row_entries(rp, rows):
    """Indices of the nonzeros of the given CSR rows, row after row."""
    rows = np.asarray(rows, dtype=np.int64)
    return np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows]) if len(rows) else np.zeros(0, np.int64)


def check_rows(rp, ci, vals, ref, rows, prec, label, m=1, base=0):
    """GPU CSR rows (numpy) against the oracle's complete rows; m dofs per vertex; the
    GPU rows start at row base (a mesh inside a batch) and columns are shifted by it."""
    dof_rows = (m * np.asarray(rows, dtype=np.int64)[:, None] + np.arange(m)[None, :]).ravel()
    got = row_entries(rp, dof_rows + base)
    want = row_entries(ref["row_ptr"], dof_rows)
    np.testing.assert_array_equal(np.diff(rp)[dof_rows + base], np.diff(ref["row_ptr"])[dof_rows])
    np.testing.assert_array_equal(ci[got] - base, ref["col_idx"][want])
    check_values(vals[got], ref, prec, label, sl=want)


@pytest.fixture(scope="module")
def headline():
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(100, seed=0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    return fe, m, q, me


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_headline_stiffness_sampled_rows_and_identities(headline, prec):
    # 3D Kuhn cube N=100, 6,000,000 tets, on the pattern the autotuner picks for the form
    fe, m, q, me = headline
    import torch
    from paper_1401_3301_gb300 import tune
    p = tune.tuned_pattern(q, me, "stiff", prec)
    vals = fe.fe_assemble_stiff(p, q, prec=prec)
    assert p.status() == (0, -1)
    rp, ci = (t.cpu().numpy() for t in p.csr())
    v = vals.double().cpu().numpy()
    rows = np.random.default_rng(1).choice(m.nq, 300, replace=False)
    keep = sub_mesh_rows(m.me, rows, m.nq)
    ref = oracle.assemble(oracle.STIFF, m.q, np.ascontiguousarray(m.me[:, keep]))
    check_rows(rp, ci, v, ref, rows, prec, "3D N=100 stiffness, sampled rows")
    # S 1 = 0 and u^T S u = |a|^2 |Omega| for u = a.x + c (exact for P1 on the unit cube)
    A = torch.sparse_csr_tensor(torch.from_numpy(rp).long(), torch.from_numpy(ci).long(), torch.from_numpy(v),
                                size=(p.n, p.n))
    scale = np.abs(v).max()
    assert float((A @ torch.ones(p.n, 1, dtype=torch.float64)).abs().max()) <= (1e-11 if prec != 1 else 1e-4) * scale
    a = np.array([0.3, -1.2, 0.7])
    u = torch.from_numpy(a @ m.q + 0.4).unsqueeze(1)
    uSu = float(u.T @ (A @ u))
    assert uSu == pytest.approx(float(a @ a), rel=1e-10 if prec != 1 else 2e-3)


def test_headline_whole_pattern_bit_exact(headline):
    # the whole CSR pattern of the 6,000,000-tet mesh (15,210,901 nonzeros, a 5-pass radix
    # sort of 40-bit keys) against the oracle's sorted-key pattern, on the pattern the
    # autotuner picks for each form (the CSR does not depend on the chunk plan)
    fe, m, q, me = headline
    from paper_1401_3301_gb300 import tune
    rp_ref, ci_ref = oracle.pattern(m.me, m.nq)
    assert len(ci_ref) == 15_210_901
    for prec in (0, 1, 2):
        p = tune.tuned_pattern(q, me, "stiff", prec)
        rp, ci = (t.cpu().numpy() for t in p.csr())
        np.testing.assert_array_equal(rp.astype(np.int64), rp_ref)
        np.testing.assert_array_equal(ci, ci_ref)


def test_elasticity_n80_whole_pattern_bit_exact():
    # 3,072,000 tets, m = 3: 70,336,089 nonzeros in 3 x 3 blocks
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(80, seed=0)
    p = fe.fe_pattern(to_cuda(m.q), to_cuda(m.me), m=3)
    rp_ref, ci_ref = oracle.pattern(m.me, m.nq, 3)
    assert len(ci_ref) == 70_336_089
    rp, ci = (t.cpu().numpy() for t in p.csr())
    np.testing.assert_array_equal(rp.astype(np.int64), rp_ref)
    np.testing.assert_array_equal(ci, ci_ref)


def test_headline_mass_and_weighted_mass_sampled_rows(headline):
    fe, m, q, me = headline
    import torch
    p = fe.fe_pattern(q, me)
    rows = np.random.default_rng(2).choice(m.nq, 200, replace=False)
    keep = sub_mesh_rows(m.me, rows, m.nq)
    sub = np.ascontiguousarray(m.me[:, keep])
    wv = meshgen.vertex_weights(0, m.nq)
    rp, ci = (t.cpu().numpy() for t in p.csr())
    for prec in (0, 1):
        T = torch.float64 if prec == 0 else torch.float32
        mass = fe.fe_assemble_mass(p, q, prec=prec).double().cpu().numpy()
        check_rows(rp, ci, mass, oracle.assemble(oracle.MASS, m.q, sub), rows, prec, "3D N=100 mass, sampled rows")
        assert mass.sum() == pytest.approx(1.0, rel=1e-12 if prec == 0 else 1e-5)  # 1^T M 1 = |Omega|
        wm = fe.fe_assemble_wmass(p, q, to_cuda(wv).to(T), fe.COEF_P1, prec=prec).double().cpu().numpy()
        check_rows(rp, ci, wm, oracle.assemble(oracle.WMASS, m.q, sub, c1=(oracle.COEF_P1, wv)), rows, prec,
                   "3D N=100 weighted mass P1, sampled rows")


@pytest.mark.parametrize("prec", [0, 1])
def test_elasticity_n80_sampled_rows(prec):
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(80, seed=0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, m=3)
    lam0, mu0 = meshgen.lame_from_young(1.0, 0.3)
    T = torch.float64 if prec == 0 else torch.float32
    lam = torch.tensor([lam0], dtype=T, device="cuda")
    mu = torch.tensor([mu0], dtype=T, device="cuda")
    vals = fe.fe_assemble_elas(p, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR, prec=prec).double().cpu().numpy()
    assert p.status() == (0, -1)
    rows = np.random.default_rng(3).choice(m.nq, 100, replace=False)
    keep = sub_mesh_rows(m.me, rows, m.nq)
    ref = oracle.assemble(oracle.ELAS, m.q, np.ascontiguousarray(m.me[:, keep]), c1=lam0, c2=mu0)
    rp, ci = (t.cpu().numpy() for t in p.csr())
    check_rows(rp, ci, vals, ref, rows, prec, "3D N=80 elasticity, sampled rows", m=3)


def test_differentiation_n64_against_oracle_gradients():
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(64, seed=0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    w = meshgen.element_weights(0, m.nme)
    u, v = meshgen.random_vectors(0, m.nq)
    Lr, dwr, dqr = oracle.stiff_loss(m.q, m.me, w, u, v)
    L = torch.empty(1, dtype=torch.float64, device="cuda")
    dw = torch.empty(m.nme, dtype=torch.float64, device="cuda")
    dq = torch.empty((3, m.nq), dtype=torch.float64, device="cuda")
    fe.fe_assemble_stiff_backward(p, q, to_cuda(w), fe.COEF_P0, to_cuda(u), to_cuda(v), L, dw, dq)
    assert p.status() == (0, -1)
    nw = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    assert nw(dw.cpu().numpy(), dwr) <= 1e-12
    assert nw(dq.cpu().numpy(), dqr) <= 1e-12
    assert abs(L.item() - Lr) <= 1e-12 * np.abs(dwr * w).sum()


def test_2d_n100_whole_matrices():
    fe = fe_or_skip()
    m = meshgen.square_mesh(100, seed=0)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    for kind, fn in ((oracle.MASS, lambda prec: fe.fe_assemble_mass(p, q, prec=prec)),
                     (oracle.STIFF, lambda prec: fe.fe_assemble_stiff(p, q, prec=prec))):
        ref = oracle.assemble(kind, m.q, m.me)
        for prec in (0, 1):
            check_values(fn(prec).double().cpu().numpy(), ref, prec,
                         "2D N=100 " + ("mass" if kind == oracle.MASS else "stiffness") + ", whole matrix")


def test_batch_of_256_meshes_sampled_meshes():
    # the 256-mesh batch of the benchmark (N uniform in [16, 512], 51.1M triangles); the
    # four smallest meshes whole, and sampled rows of the largest
    fe = fe_or_skip()
    import torch
    sizes = meshgen.batch_sizes(0, 256, 16, 512)
    meshes = [meshgen.square_mesh(int(n), seed=b + 1) for b, n in enumerate(sizes)]
    qs = [to_cuda(x.q) for x in meshes]
    mes = [to_cuda(x.me) for x in meshes]
    p = fe.fe_batch_pattern(qs, mes)
    vo, eo, no = fe.fe_batch_offsets(p)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p, qs, mes, qu)
    del qs, mes
    ws = [meshgen.element_weights(100 + b, x.nme) for b, x in enumerate(meshes)]
    s = fe.fe_assemble_stiff(p, qu, to_cuda(np.concatenate(ws)), fe.COEF_P0).cpu().numpy()
    assert p.status() == (0, -1)
    rp, ci = (t.cpu().numpy() for t in p.csr())
    order = np.argsort(sizes)
    for b in order[:4]:
        x = meshes[b]
        ref = oracle.assemble(oracle.STIFF, x.q, x.me, c1=(oracle.COEF_P0, ws[b]))
        sl = slice(int(no[b]), int(no[b + 1]))
        np.testing.assert_array_equal(ci[sl] - vo[b], ref["col_idx"])
        check_values(s[sl], ref, 0, "2D batch of 256: smallest meshes whole")
    b = order[-1]
    x = meshes[b]
    rows = np.random.default_rng(4).choice(x.nq, 200, replace=False)
    keep = sub_mesh_rows(x.me, rows, x.nq)
    ref = oracle.assemble(oracle.STIFF, x.q, np.ascontiguousarray(x.me[:, keep]), c1=(oracle.COEF_P0, ws[b][keep]))
    check_rows(rp, ci, s, ref, rows, 0, "2D batch of 256: largest mesh, sampled rows", base=int(vo[b]))


def test_surface_n2000_boundary_mass_sampled_rows():
    # the facet workload of the benchmark: 8,000,000 triangles in 3D
    fe = fe_or_skip()
    import torch
    m = meshgen.surface_mesh(2000, seed=0)
    q, f = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_boundary_pattern(q, f)
    wv = meshgen.vertex_weights(0, m.nq)
    rows = np.random.default_rng(5).choice(m.nq, 200, replace=False)
    keep = sub_mesh_rows(m.me, rows, m.nq)
    sub = np.ascontiguousarray(m.me[:, keep])
    rp, ci = (t.cpu().numpy() for t in p.csr())
    for prec in (0, 1):
        T = torch.float64 if prec == 0 else torch.float32
        mass = fe.fe_assemble_mass(p, q, prec=prec).double().cpu().numpy()
        check_rows(rp, ci, mass, oracle.assemble_boundary(oracle.MASS, m.q, sub), rows, prec,
                   "surface N=2000 facet mass, sampled rows")
        wm = fe.fe_assemble_wmass(p, q, to_cuda(wv).to(T), fe.COEF_P1, prec=prec).double().cpu().numpy()
        check_rows(rp, ci, wm, oracle.assemble_boundary(oracle.WMASS, m.q, sub, c1=(oracle.COEF_P1, wv)), rows,
                   prec, "surface N=2000 facet weighted mass P1, sampled rows")
        assert p.status() == (0, -1)

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU. Each check is chosen so that a plausible slip in the oracle (a dropped
term, a sign, a transposed index, a wrong factorial) fails at least one of them.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import exact_p1_matrices

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def duffy_rule(d, n=8):
    """Collapsed-coordinate Gauss-Legendre rule on the reference simplex (independent quadrature)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    pts, wts = [], []
    if d == 2:
        for (u, wu), (v, wv) in itertools.product(zip(x, w), zip(x, w)):
            pts.append((u, v * (1 - u)))
            wts.append(wu * wv * (1 - u))
    else:
        for (u, wu), (v, wv), (t, wt) in itertools.product(zip(x, w), zip(x, w), zip(x, w)):
            pts.append((u, v * (1 - u), t * (1 - u) * (1 - v)))
            wts.append(wu * wv * wt * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def bary_ref(pts):
    """Barycentric coordinates on the reference simplex: lambda_0 = 1 - sum x, lambda_i = x_i."""
    return np.column_stack([1.0 - pts.sum(axis=1), pts])


def random_simplex(rng, d):
    while True:
        X = rng.normal(size=(d + 1, d))
        if abs(np.linalg.det((X[1:] - X[0]).T)) > 0.2:
            return X


def read_golden(name):
    verts, elems, entries = [], [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "vertex":
                verts.append([float(t) for t in line[2:]])
            elif line[0] == "element":
                elems.append([int(t) for t in line[1:]])
            else:
                val = sum(Fraction(t) for t in line[3].split("+"))
                entries.setdefault(line[0], {})[(int(line[1]), int(line[2]))] = float(val)
    q = np.array(verts).T.copy()
    me = np.array(elems, dtype=np.int32).T.copy()
    return q, me, entries


def csr_entries(res):
    rows = np.repeat(np.arange(res["n"]), np.diff(res["row_ptr"]))
    return {(int(r), int(c)): v for r, c, v in zip(rows, res["col_idx"], res["val"])}


# ---------------------------------------------------------------- magic formula and geometry
@pytest.mark.parametrize("d", [2, 3])
def test_magic_formula_against_quadrature(d):
    rng = np.random.default_rng(1)
    X = random_simplex(rng, d)
    det, vol, _ = oracle.simplex(X)
    pts, wts = duffy_rule(d)
    lam = bary_ref(pts)
    for n in itertools.product(range(3), repeat=d + 1):
        if sum(n) > 4:
            continue
        quad = abs(det) * np.sum(wts * np.prod(lam ** np.array(n), axis=1))
        assert oracle.magic(d, n, vol) == pytest.approx(quad, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_simplex_gradients_are_barycentric(d):
    rng = np.random.default_rng(2)
    for _ in range(20):
        X = random_simplex(rng, d)
        det, vol, G = oracle.simplex(X)
        B = (X[1:] - X[0]).T
        assert det == pytest.approx(np.linalg.det(B), rel=1e-12)
        assert vol == pytest.approx(abs(np.linalg.det(B)) / (2 if d == 2 else 6), rel=1e-12)
        # lambda_a is affine with lambda_a(X_b) = delta_ab, so G_a . (X_b - X_c) = delta_ab - delta_ac
        for a, b, c in itertools.product(range(d + 1), repeat=3):
            lhs = G[a] @ (X[b] - X[c])
            assert lhs == pytest.approx(float(a == b) - float(a == c), abs=1e-11)
        assert np.abs(G.sum(axis=0)).max() < 1e-11


def test_unit_right_simplices_stiffness():
    # textbook element matrices of the reference triangle / tetrahedron
    Et, _ = oracle.element(oracle.STIFF, np.array([[0, 0], [1, 0], [0, 1]], float))
    np.testing.assert_allclose(Et, 0.5 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]]), atol=1e-15)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    Ek, _ = oracle.element(oracle.STIFF, X)
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    np.testing.assert_allclose(Ek, ref, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_mass_closed_form(d):
    # Section 4.1 with w = 1: |K| d!/(d+2)! (1 + delta), i.e. |K|/12 (2D), |K|/20 (3D)
    rng = np.random.default_rng(3)
    X = random_simplex(rng, d)
    _, vol, _ = oracle.simplex(X)
    E, _ = oracle.element(oracle.MASS, X)
    c = 12.0 if d == 2 else 20.0
    np.testing.assert_allclose(E, vol / c * (1 + np.eye(d + 1)), rtol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_weighted_mass_closed_form_and_quadrature(d):
    rng = np.random.default_rng(4)
    X = random_simplex(rng, d)
    det, vol, _ = oracle.simplex(X)
    w = rng.uniform(0.5, 2.0, size=d + 1)
    E, _ = oracle.element(oracle.WMASS, X, cv1=w)
    # Eq. MatElemMassWP1: d!/(d+3)! |K| (1 + delta_ab)(w^s + w_a + w_b)
    fac = (2.0 if d == 2 else 6.0) / (120.0 if d == 2 else 720.0)
    closed = fac * vol * (1 + np.eye(d + 1)) * (w.sum() + w[:, None] + w[None, :])
    np.testing.assert_allclose(E, closed, rtol=1e-13)
    # independent: quadrature of (sum_g w_g lambda_g) lambda_a lambda_b (cubic -> exact)
    pts, wts = duffy_rule(d)
    lam = bary_ref(pts)
    wh = lam @ w
    quad = abs(det) * np.einsum("p,p,pa,pb->ab", wts, wh, lam, lam)
    np.testing.assert_allclose(E, quad, rtol=1e-12)


# ---------------------------------------------------------------- golden two-element meshes
@pytest.mark.parametrize("name", ["two_triangles.txt", "two_tets.txt"])
def test_two_element_golden(name):
    q, me, gold = read_golden(name)
    for kind, key in ((oracle.STIFF, "stiff"), (oracle.MASS, "mass")):
        res = oracle.assemble(kind, q, me)
        got = csr_entries(res)
        assert set(got) == set(gold[key]), key  # pattern, including the structural zeros
        for ij, v in gold[key].items():
            assert got[ij] == pytest.approx(v, abs=1e-15), (key, ij)


# ---------------------------------------------------------------- global invariants
def test_global_mass_and_stiffness_invariants_2d():
    m = meshgen.square_mesh(12, seed=5)
    x, y = m.q
    M = oracle.to_dense(oracle.assemble(oracle.MASS, m.q, m.me))
    S = oracle.to_dense(oracle.assemble(oracle.STIFF, m.q, m.me))
    one = np.ones(m.nq)
    assert one @ M @ one == pytest.approx(1.0, rel=1e-13)       # |Omega|
    assert x @ M @ x == pytest.approx(1.0 / 3.0, rel=1e-13)     # int x^2 (P1 exact)
    assert x @ M @ y == pytest.approx(1.0 / 4.0, rel=1e-13)     # int x y
    assert np.abs(S @ one).max() < 1e-13
    a, c = np.array([0.7, -1.3]), 0.4
    u = a @ m.q + c
    assert u @ S @ u == pytest.approx(a @ a, rel=1e-12)          # |a|^2 |Omega|
    np.testing.assert_allclose(S, S.T, atol=1e-14)
    assert np.linalg.eigvalsh(S).min() > -1e-12


def test_global_invariants_3d_and_weighted_mass():
    m = meshgen.kuhn_cube_mesh(4, seed=6)
    one = np.ones(m.nq)
    M = oracle.to_dense(oracle.assemble(oracle.MASS, m.q, m.me))
    assert one @ M @ one == pytest.approx(1.0, rel=1e-13)
    x, y, z = m.q
    assert z @ M @ z == pytest.approx(1.0 / 3.0, rel=1e-12)
    S = oracle.to_dense(oracle.assemble(oracle.STIFF, m.q, m.me))
    assert np.abs(S @ one).max() < 1e-13
    a = np.array([0.3, -0.8, 1.1])
    u = a @ m.q
    assert u @ S @ u == pytest.approx(a @ a, rel=1e-12)
    # P1 weight w = 2 + x - y + 3z: the P1 rule is exact, 1^T M_w 1 = int w = 2 + 0.5 - 0.5 + 1.5
    w = 2 + x - y + 3 * z
    Mw = oracle.to_dense(oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P1, w)))
    assert one @ Mw @ one == pytest.approx(3.5, rel=1e-13)
    # int w x = int (2x + x^2 - xy + 3xz) = 1 + 1/3 - 1/4 + 3/4
    assert one @ Mw @ x == pytest.approx(1 + 1 / 3 - 1 / 4 + 3 / 4, rel=1e-12)
    # P0 weight: 1^T M 1 = sum_K w_K |K|
    wk = meshgen.element_weights(6, m.nme)
    M0 = oracle.assemble(oracle.WMASS, m.q, m.me, c1=(oracle.COEF_P0, wk))
    vols = np.array([oracle.simplex(m.q[:, m.me[:, k]].T)[1] for k in range(m.nme)])
    assert M0["val"].sum() == pytest.approx((wk * vols).sum(), rel=1e-13)


# ---------------------------------------------------------------- elasticity
def paper_QS(d):
    """Q^{n,l} = B_n^T C0 B_l and S^{n,l} = B_n^T C1 B_l with B_l, C0, C1 as printed in App. B."""
    def Bl(l):
        dl = [float(l == i) for i in range(d)]
        if d == 2:
            return np.array([[dl[0], 0], [0, dl[1]], [dl[1], dl[0]]])
        return np.array([[dl[0], 0, 0], [0, dl[1], 0], [0, 0, dl[2]],
                         [dl[1], dl[0], 0], [0, dl[2], dl[1]], [dl[2], 0, dl[0]]])
    ns = 3 * (d - 1)
    C0 = np.zeros((ns, ns))
    C0[:d, :d] = 1.0
    C1 = np.diag([2.0] * d + [1.0] * (ns - d))
    Q = {(n, l): Bl(n).T @ C0 @ Bl(l) for n in range(d) for l in range(d)}
    S = {(n, l): Bl(n).T @ C1 @ Bl(l) for n in range(d) for l in range(d)}
    return Q, S


@pytest.mark.parametrize("d", [2, 3])
def test_elasticity_element_matches_lemma(d):
    # Lemma (Section 5.1): eps(phi_{n,b})^T C eps(phi_{l,a}) = lam <g_b, Q^{n,l} g_a> + mu <g_b, S^{n,l} g_a>
    rng = np.random.default_rng(7)
    X = random_simplex(rng, d)
    _, vol, G = oracle.simplex(X)
    lam_v, mu_v = rng.uniform(0.5, 2, d + 1), rng.uniform(0.5, 2, d + 1)
    E, _ = oracle.element(oracle.ELAS, X, cv1=lam_v, cv2=mu_v)
    Q, S = paper_QS(d)
    lam_s, mu_s = vol / (d + 1) * lam_v.sum(), vol / (d + 1) * mu_v.sum()
    for a, l, b, n in itertools.product(range(d + 1), range(d), range(d + 1), range(d)):
        ref = lam_s * G[b] @ Q[(n, l)] @ G[a] + mu_s * G[b] @ S[(n, l)] @ G[a]
        assert E[a * d + l, b * d + n] == pytest.approx(ref, rel=1e-12, abs=1e-14)
    # and the closed forms Q^{n,l} = e_n e_l^T, S^{n,l} = delta_nl I + e_l e_n^T
    I = np.eye(d)
    for n, l in itertools.product(range(d), range(d)):
        np.testing.assert_array_equal(Q[(n, l)], np.outer(I[n], I[l]))
        np.testing.assert_array_equal(S[(n, l)], (n == l) * I + np.outer(I[l], I[n]))


def rigid_modes(q):
    d = q.shape[0]
    modes = []
    for c in range(d):
        u = np.zeros((q.shape[1], d))
        u[:, c] = 1.0
        modes.append(u.ravel())
    if d == 2:
        modes.append(np.column_stack([-q[1], q[0]]).ravel())
    else:
        for axis in range(3):
            w = np.zeros(3)
            w[axis] = 1.0
            modes.append(np.cross(w, q.T).ravel())
    return modes


@pytest.mark.parametrize("d", [2, 3])
def test_elasticity_rigid_modes_and_patch(d):
    m = meshgen.square_mesh(6, seed=8) if d == 2 else meshgen.kuhn_cube_mesh(3, seed=8)
    lam, mu = meshgen.lame_from_young(1.0, 0.3)
    K = oracle.to_dense(oracle.assemble(oracle.ELAS, m.q, m.me, c1=lam, c2=mu))
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    for u in rigid_modes(m.q):
        assert np.abs(K @ u).max() < 1e-12
    assert np.linalg.eigvalsh(K).min() > -1e-11
    # patch test with a non-symmetric A of nonzero trace: u = A x has constant strain sym(A)
    rng = np.random.default_rng(9)
    A = rng.normal(size=(d, d))
    u = (A @ m.q).T.ravel()  # alternate numbering: dof = d * vertex + component
    epsA = 0.5 * (A + A.T)
    energy = lam * np.trace(A) ** 2 + 2 * mu * np.sum(epsA * epsA)  # times |Omega| = 1
    assert u @ K @ u == pytest.approx(energy, rel=1e-11)


# ---------------------------------------------------------------- pattern
@pytest.mark.parametrize("d", [2, 3])
def test_pattern_brute_force(d):
    m = meshgen.square_mesh(5, seed=10) if d == 2 else meshgen.kuhn_cube_mesh(2, seed=10)
    res = oracle.assemble(oracle.STIFF, m.q, m.me)
    adj = np.zeros((m.nq, m.nq), bool)
    for k in range(m.nme):
        for a in m.me[:, k]:
            for b in m.me[:, k]:
                adj[a, b] = True
    r, c = np.nonzero(adj)  # row-major, sorted columns
    assert res["nnz"] == len(r)
    np.testing.assert_array_equal(np.repeat(np.arange(m.nq), np.diff(res["row_ptr"])), r)
    np.testing.assert_array_equal(res["col_idx"], c)
    edges = {tuple(sorted((int(a), int(b)))) for k in range(m.nme)
             for a, b in itertools.combinations(m.me[:, k], 2)}
    assert res["nnz"] == m.nq + 2 * len(edges)
    # vector case: 3x3 / 2x2 blocks in the alternate numbering
    lam, mu = meshgen.lame_from_young(1.0, 0.3)
    re = oracle.assemble(oracle.ELAS, m.q, m.me, c1=lam, c2=mu)
    assert re["nnz"] == d * d * res["nnz"]


@pytest.mark.parametrize("d,m_dofs", [(2, 1), (2, 2), (3, 1), (3, 3)])
def test_pattern_alone_against_dense_adjacency(d, m_dofs):
    # oracle.pattern (sorted keys, no values) against a dense boolean adjacency and, for
    # vector unknowns, its Kronecker product with an m x m block of ones
    m = meshgen.square_mesh(6, seed=31) if d == 2 else meshgen.kuhn_cube_mesh(3, seed=31)
    rp, ci = oracle.pattern(m.me, m.nq, m_dofs)
    adj = np.zeros((m.nq, m.nq), bool)
    for k in range(m.nme):
        adj[np.ix_(m.me[:, k], m.me[:, k])] = True
    big = np.kron(adj, np.ones((m_dofs, m_dofs), bool))
    r, c = np.nonzero(big)
    np.testing.assert_array_equal(np.repeat(np.arange(m_dofs * m.nq), np.diff(rp)), r)
    np.testing.assert_array_equal(ci, c)
    # the same pattern as the full assembly's `sparse` step
    kind, cs = (oracle.STIFF, ()) if m_dofs == 1 else (oracle.ELAS, (0.5, 0.3))
    res = oracle.assemble(kind, m.q, m.me, *cs)
    np.testing.assert_array_equal(rp, res["row_ptr"])
    np.testing.assert_array_equal(ci, res["col_idx"])


@pytest.mark.parametrize("d,N", [(2, 6), (3, 3)])
def test_values_against_exact_rational_arithmetic(d, N):
    # the oracle's FP64 sums against the exactly computed matrices of the same (double)
    # coordinates: errors within a few units of rounding of the normwise scale, and the
    # sum of |contributions| (the condition scale of each entry) reproduced exactly
    m = meshgen.square_mesh(N, seed=33) if d == 2 else meshgen.kuhn_cube_mesh(N, seed=33)
    ex = exact_p1_matrices(m.q, m.me)
    rs = oracle.assemble(oracle.STIFF, m.q, m.me)
    rm = oracle.assemble(oracle.MASS, m.q, m.me)
    rows = np.repeat(np.arange(rs["n"]), np.diff(rs["row_ptr"]))
    keys = list(zip(rows.tolist(), rs["col_idx"].tolist()))
    assert set(keys) == set(ex)
    s_ex = np.array([float(ex[k][0]) for k in keys])
    m_ex = np.array([float(ex[k][1]) for k in keys])
    a_ex = np.array([float(ex[k][2]) for k in keys])
    u = 2.0 ** -53
    assert np.all(np.abs(rs["val"] - s_ex) <= 64 * u * rs["scale"])
    assert np.all(np.abs(rs["abssum"] - a_ex) <= 64 * u * rs["scale"])
    assert np.all(np.abs(rm["val"] - m_ex) <= 8 * u * np.abs(m_ex))
    # per entry against the sum of |contributions|: the oracle itself meets the FP64 gate
    # (entries whose every contribution is exactly zero are exactly zero on both sides)
    zero = a_ex == 0
    assert np.all(rs["val"][zero] == 0) and np.all(rs["abssum"][zero] == 0)
    assert np.max(np.abs(rs["val"] - s_ex)[~zero] / a_ex[~zero]) <= 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_fixed_pattern_reassembly_and_threads(d):
    # the slot map's sums reproduce orc_assemble bit for bit, and neither the threaded
    # element loops nor the threaded sort change a bit (where the build has OpenMP)
    m = meshgen.square_mesh(9, seed=34) if d == 2 else meshgen.kuhn_cube_mesh(4, seed=34)
    w = meshgen.element_weights(34, m.nme)
    ref = oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, w))
    ptr, n2s = oracle.slot_map(m.me, m.nq)
    assert len(ptr) == ref["nnz"] + 1 and sorted(n2s.tolist()) == list(range(m.nme * (d + 1) ** 2))
    # the slots of each nonzero name that (row, column): slot k ns + b (d+1) + a is (me[a,k], me[b,k])
    nv = d + 1
    k, loc = n2s // nv ** 2, n2s % nv ** 2
    rows_of_slot = m.me[loc % nv, k]
    cols_of_slot = m.me[loc // nv, k]
    rows = np.repeat(np.arange(ref["n"]), np.diff(ref["row_ptr"]))
    np.testing.assert_array_equal(rows_of_slot, np.repeat(rows, np.diff(ptr)))
    np.testing.assert_array_equal(cols_of_slot, np.repeat(ref["col_idx"], np.diff(ptr)))
    try:
        for threads in (1, 4):
            oracle.set_threads(threads)
            v = oracle.reassemble(oracle.STIFF, m.q, m.me, ptr, n2s, c1=(oracle.COEF_P0, w))
            np.testing.assert_array_equal(v, ref["val"])
            r2 = oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, w))
            for key in ("row_ptr", "col_idx", "val", "scale", "abssum"):
                np.testing.assert_array_equal(r2[key], ref[key])
            p2, s2 = oracle.slot_map(m.me, m.nq)
            np.testing.assert_array_equal(p2, ptr)
            np.testing.assert_array_equal(s2, n2s)
        bad = m.me.copy()
        bad[1, 5] = m.nq + 3
        with pytest.raises(oracle.OracleError) as e:
            oracle.assemble(oracle.STIFF, m.q, bad)
        assert e.value.code == 2 and e.value.bad_id == 5
    finally:
        oracle.set_threads(1)


# ---------------------------------------------------------------- derivatives
@pytest.mark.parametrize("d", [2, 3])
def test_stiffness_loss_gradients(d):
    m = meshgen.square_mesh(5, seed=11) if d == 2 else meshgen.kuhn_cube_mesh(2, seed=11)
    w = meshgen.element_weights(11, m.nme)
    u, v = meshgen.random_vectors(11, m.nq)
    L, dw, dq = oracle.stiff_loss(m.q, m.me, w, u, v)
    # L equals u^T K(w) v with the assembled matrix
    K = oracle.to_dense(oracle.assemble(oracle.STIFF, m.q, m.me, c1=(oracle.COEF_P0, w)))
    assert L == pytest.approx(u @ K @ v, rel=1e-12)
    # L is linear in w: dL/dw_e times w_e sums to L
    assert np.dot(dw, w) == pytest.approx(L, rel=1e-12)
    # central differences in q and w
    rng = np.random.default_rng(12)
    h = 1e-6
    for _ in range(12):
        c, vtx = rng.integers(d), rng.integers(m.nq)
        qp, qm = m.q.copy(), m.q.copy()
        qp[c, vtx] += h
        qm[c, vtx] -= h
        fd = (oracle.stiff_loss(qp, m.me, w, u, v, False)[0] - oracle.stiff_loss(qm, m.me, w, u, v, False)[0]) / (2 * h)
        assert dq[c, vtx] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(dq).max())
    # invariances: translation (sum of dL/dq = 0) and rotation (sum q x dL/dq = 0)
    assert np.abs(dq.sum(axis=1)).max() < 1e-11 * np.abs(dq).max() * m.nq
    if d == 2:
        torque = np.sum(m.q[0] * dq[1] - m.q[1] * dq[0])
        assert abs(torque) < 1e-11 * np.abs(dq).max() * m.nq
    else:
        torque = np.cross(m.q.T, dq.T).sum(axis=0)
        assert np.abs(torque).max() < 1e-11 * np.abs(dq).max() * m.nq


# ---------------------------------------------------------------- errors
def test_oracle_reports_bad_input():
    m = meshgen.square_mesh(3, seed=0)
    me = m.me.copy()
    me[1, 5] = m.nq
    with pytest.raises(oracle.OracleError) as e:
        oracle.assemble(oracle.STIFF, m.q, me)
    assert e.value.code == 2 and e.value.bad_id == 5
    q = m.q.copy()
    a, b, c = m.me[:, 7]
    q[:, c] = 0.5 * (q[:, a] + q[:, b])  # collapse element 7 (and maybe neighbours)
    with pytest.raises(oracle.OracleError) as e:
        oracle.assemble(oracle.STIFF, q, m.me)
    assert e.value.code == 3


# ---------------------------------------------------------------- boundary (facet) mass
def test_facet_measure_against_heron_and_length():
    rng = np.random.default_rng(20)
    for _ in range(10):
        X = rng.normal(size=(3, 3))
        a, b, c = (np.linalg.norm(X[i] - X[j]) for i, j in ((0, 1), (1, 2), (2, 0)))
        s = 0.5 * (a + b + c)
        heron = np.sqrt(s * (s - a) * (s - b) * (s - c))
        assert oracle.facet_measure(X) == pytest.approx(heron, rel=1e-10)
        Y = rng.normal(size=(2, 2))
        assert oracle.facet_measure(Y) == pytest.approx(np.hypot(*(Y[1] - Y[0])), rel=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_boundary_mass_integrals(d):
    m = meshgen.square_mesh(7, seed=21) if d == 2 else meshgen.kuhn_cube_mesh(4, seed=21)
    fa = meshgen.boundary_facets(m)
    M = oracle.to_dense(oracle.assemble_boundary(oracle.MASS, m.q, fa))
    one = np.ones(m.nq)
    x = m.q[0]
    assert one @ M @ one == pytest.approx(4.0 if d == 2 else 6.0, rel=1e-13)          # perimeter / area
    assert x @ M @ x == pytest.approx(5.0 / 3.0 if d == 2 else 7.0 / 3.0, rel=1e-12)  # int x^2 ds
    # P1 weight w = 1 + x is integrated exactly: int (1 + x) ds = 6 (square), 6 + 3 (cube)
    Mw = oracle.to_dense(oracle.assemble_boundary(oracle.WMASS, m.q, fa, c1=(oracle.COEF_P1, 1.0 + x)))
    assert one @ Mw @ one == pytest.approx(6.0 if d == 2 else 9.0, rel=1e-12)
    # element closed forms: segment |K|/6 (1 + delta), triangle |K|/12 (1 + delta)
    X = m.q[:, fa[:, 0]].T
    _, meas = None, oracle.facet_measure(X)
    single = oracle.to_dense(oracle.assemble_boundary(oracle.MASS, m.q, fa[:, :1]))
    idx = fa[:, 0]
    np.testing.assert_allclose(single[np.ix_(idx, idx)], meas / (6.0 if d == 2 else 12.0) * (1 + np.eye(d)),
                               rtol=1e-14)


# ---------------------------------------------------------------- general operator (Eq. EDP)
def general_coef(d, A, b, c, a0):
    return np.concatenate([np.asarray(A, float).ravel(), b, c, [a0]])


@pytest.mark.parametrize("d", [2, 3])
def test_general_operator_reduces_to_stiffness_and_mass(d):
    m = meshgen.square_mesh(6, seed=30) if d == 2 else meshgen.kuhn_cube_mesh(3, seed=30)
    z = np.zeros(d)
    S = oracle.to_dense(oracle.assemble(oracle.STIFF, m.q, m.me))
    G = oracle.to_dense(oracle.assemble_general(m.q, m.me, general_coef(d, np.eye(d), z, z, 0.0), oracle.COEF_SCALAR))
    np.testing.assert_allclose(G, S, atol=1e-14)
    M = oracle.to_dense(oracle.assemble(oracle.MASS, m.q, m.me))
    G0 = oracle.to_dense(oracle.assemble_general(m.q, m.me, general_coef(d, np.zeros((d, d)), z, z, 2.5), oracle.COEF_SCALAR))
    np.testing.assert_allclose(G0, 2.5 * M, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_general_operator_bilinear_form_on_linear_functions(d):
    # v^T M u = a(u, v) exactly for P1 u = alpha.x + alpha0, v = gamma.x + gamma0 (polynomial
    # integrands of degree <= 2 over the unit square / cube)
    m = meshgen.square_mesh(5, seed=31) if d == 2 else meshgen.kuhn_cube_mesh(3, seed=31)
    rng = np.random.default_rng(32)
    A, bv, cv, a0 = rng.normal(size=(d, d)), rng.normal(size=d), rng.normal(size=d), 0.7
    M = oracle.to_dense(oracle.assemble_general(m.q, m.me, general_coef(d, A, bv, cv, a0), oracle.COEF_SCALAR))
    al, al0, ga, ga0 = rng.normal(size=d), 0.3, rng.normal(size=d), -0.4
    u = al @ m.q + al0
    v = ga @ m.q + ga0
    mean_u = al.sum() / 2 + al0          # int_Omega u over the unit cube/square
    mean_v = ga.sum() / 2 + ga0
    Exx = np.full((d, d), 0.25) + np.eye(d) * (1 / 3 - 0.25)   # int x_i x_j
    int_uv = al @ Exx @ ga + al0 * ga.sum() / 2 + ga0 * al.sum() / 2 + al0 * ga0
    exact = (A @ al) @ ga - (bv @ ga) * mean_u + (cv @ al) * mean_v + a0 * int_uv
    assert v @ M @ u == pytest.approx(exact, rel=1e-12)
    # transposed orientation would differ: the operator is not symmetric
    assert abs(u @ M @ v - exact) > 1e-6


def test_general_operator_per_element_coefficients():
    # constant per-element columns equal the scalar form; the matrix is linear in each
    # element's coefficients, so two halves of a coefficient field add up
    m = meshgen.square_mesh(5, seed=33)
    rng = np.random.default_rng(34)
    cf = general_coef(2, rng.normal(size=(2, 2)), rng.normal(size=2), rng.normal(size=2), 1.3)
    S = oracle.to_dense(oracle.assemble_general(m.q, m.me, cf, oracle.COEF_SCALAR))
    P = oracle.to_dense(oracle.assemble_general(m.q, m.me, np.repeat(cf[None, :], m.nme, 0), oracle.COEF_P0))
    np.testing.assert_allclose(P, S, atol=1e-14)
    F = rng.normal(size=(m.nme, cf.size))
    mask = (np.arange(m.nme) % 2 == 0)[:, None]
    Fa, Fb = F * mask, F * ~mask
    T = oracle.to_dense(oracle.assemble_general(m.q, m.me, F, oracle.COEF_P0))
    Ta = oracle.to_dense(oracle.assemble_general(m.q, m.me, Fa, oracle.COEF_P0))
    Tb = oracle.to_dense(oracle.assemble_general(m.q, m.me, Fb, oracle.COEF_P0))
    np.testing.assert_allclose(Ta + Tb, T, atol=1e-13)


def _gauss_cube(d, npts=3):
    """Tensor Gauss-Legendre rule on [0, 1]^d: exact for degree <= 2 npts - 1 per variable."""
    x, w = np.polynomial.legendre.leggauss(npts)
    x, w = (x + 1) / 2, w / 2
    grids = np.meshgrid(*([x] * d), indexing="ij")
    wts = np.prod(np.meshgrid(*([w] * d), indexing="ij"), axis=0)
    return np.stack([g.ravel() for g in grids]), wts.ravel()


@pytest.mark.parametrize("d", [2, 3])
def test_general_operator_p1_coefficients_by_quadrature(d):
    # Linear coefficient fields (exactly P1) and linear u, v: every integrand of a(u, v)
    # is a polynomial of degree <= 3, integrated exactly over the unit square / cube by
    # 3-point tensor Gauss quadrature, independent of the magic formula.
    m = meshgen.square_mesh(4, seed=35) if d == 2 else meshgen.kuhn_cube_mesh(3, seed=35)
    rng = np.random.default_rng(36)
    nc = d * d + 2 * d + 1
    slope, base = rng.normal(size=(nc, d)), rng.normal(size=nc)
    coef_at = lambda x: slope @ x + base[:, None]           # (nc, npoints), linear in x
    cf = coef_at(m.q).T.copy()                               # nodal records (nq, nc)
    M = oracle.to_dense(oracle.assemble_general(m.q, m.me, cf, oracle.COEF_P1))
    al, al0, ga, ga0 = rng.normal(size=d), 0.3, rng.normal(size=d), -0.4
    u, v = al @ m.q + al0, ga @ m.q + ga0
    X, W = _gauss_cube(d)
    C = coef_at(X)
    A = C[: d * d].reshape(d, d, -1)
    bq, cq, a0 = C[d * d: d * d + d], C[d * d + d: nc - 1], C[nc - 1]
    uq, vq = al @ X + al0, ga @ X + ga0
    integrand = (np.einsum("ijp,j,i->p", A, al, ga) - uq * (ga @ bq) + (al @ cq) * vq + a0 * uq * vq)
    assert v @ M @ u == pytest.approx(W @ integrand, rel=1e-12)


def test_general_operator_p1_constant_fields_match_scalar():
    m = meshgen.square_mesh(5, seed=37)
    cf = general_coef(2, [[1.0, 0.2], [-0.4, 2.0]], [0.3, -1.0], [0.5, 0.25], 1.5)
    S = oracle.to_dense(oracle.assemble_general(m.q, m.me, cf, oracle.COEF_SCALAR))
    P = oracle.to_dense(oracle.assemble_general(m.q, m.me, np.repeat(cf[None, :], m.nq, 0), oracle.COEF_P1))
    np.testing.assert_allclose(P, S, atol=1e-14)


# ---------------------------------------------------------------- P_k mass (App. D)
from fractions import Fraction  # noqa: E402


@pytest.mark.parametrize("d", [2, 3])
def test_pk_table_k1_is_the_p1_mass(d):
    t = oracle.pk_mass_table(d, 1)
    base = Fraction(math.factorial(d), math.factorial(d + 2))
    for a in range(d + 1):
        for b in range(d + 1):
            assert t[a][b] == base * (2 if a == b else 1)


def test_pk_table_p2_closed_forms():
    # P2 triangle: |K|/180 [6 on vertex diagonals, -1 vertex-vertex, -4 vertex-opposite edge,
    # 0 vertex-adjacent edge, 32 edge diagonals, 16 edge-edge]
    al = oracle.pk_multi_indices(2, 2)
    t = oracle.pk_mass_table(2, 2)
    for i, a in enumerate(al):
        for j, b in enumerate(al):
            va, vb = max(a) == 2, max(b) == 2
            if va and vb:
                want = 6 if i == j else -1
            elif va or vb:
                v, e = (a, b) if va else (b, a)
                want = -4 if all(v[x] == 0 or e[x] == 0 for x in range(3)) else 0
            else:
                want = 32 if i == j else 16
            assert t[i][j] == Fraction(want, 180), (a, b)
    # P2 tetrahedron: integral of a vertex basis function is -|K|/20, of an edge one |K|/5
    t3 = oracle.pk_mass_table(3, 2)
    for a, row in zip(oracle.pk_multi_indices(3, 2), t3):
        assert sum(row) == (Fraction(-1, 20) if max(a) == 2 else Fraction(1, 5))


@pytest.mark.parametrize("d,k", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_pk_basis_is_lagrange_on_the_lattice(d, k):
    al = oracle.pk_multi_indices(d, k)
    for a in al:
        poly = oracle._pk_basis(a, k)
        for b in al:
            lam = [Fraction(x, k) for x in b]
            val = sum(c * math.prod(l ** m for l, m in zip(lam, mu)) for mu, c in poly.items())
            assert val == (1 if a == b else 0)


@pytest.mark.parametrize("d,k", [(2, 3), (2, 5), (3, 3), (3, 4)])
def test_pk_table_symmetric_partition_of_unity(d, k):
    t = oracle.pk_mass_table(d, k)
    n = math.comb(d + k, k)
    assert len(t) == n
    assert sum(sum(r) for r in t) == 1
    assert all(t[i][j] == t[j][i] for i in range(n) for j in range(n))


@pytest.mark.parametrize("d,N,k", [(2, 3, 1), (2, 3, 2), (2, 2, 3), (2, 2, 4), (3, 2, 1), (3, 2, 2), (3, 1, 3)])
def test_pk_mass_of_polynomials_by_quadrature(d, N, k):
    # P_k contains every polynomial of degree <= k, so the nodal values of such u, v give
    # v^T M u = int u v exactly over the unit square / cube; tensor Gauss quadrature with
    # k + 1 points per direction is exact for the product (degree <= 2k per variable).
    m = meshgen.pk_mesh(d, N, k, seed=40 + k)
    rng = np.random.default_rng(41)
    exps = [e for e in np.ndindex(*([k + 1] * d)) if sum(e) <= k]
    cu, cv = rng.normal(size=len(exps)), rng.normal(size=len(exps))
    poly = lambda c, X: sum(ci * np.prod([X[j] ** e[j] for j in range(d)], axis=0) for ci, e in zip(c, exps))
    M = oracle.to_dense(oracle.assemble_pk_mass(m.q, m.me, k))
    X, W = _gauss_cube(d, k + 1)
    exact = W @ (poly(cu, X) * poly(cv, X))
    assert poly(cv, m.q) @ M @ poly(cu, m.q) == pytest.approx(exact, rel=1e-11, abs=1e-13)

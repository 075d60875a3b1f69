"""Badly shaped elements: slivers, caps and needles whose det B is 1e-2 down to 1e-10 of
the products it is formed from (App. C.1: B_k, det B_k and the barycentric gradients).

The meshes are isolated simplices (meshgen.badly_shaped_mesh), so every matrix entry is
one element's contribution and the exact values of the same (double) coordinates are
computed in rational arithmetic (helpers.exact_p1_matrices). Checked:
  - FP32 form: |K| (through the mass matrix, |det B| (1 + delta) / (d+2)!) within 1e-6
    of the exact value, and the stiffness within 1e-5 per nonzero of the exact
    contributions' normwise scale, at every flatness: the form recomputes det B in FP64
    where its double-float value is too close to its error bound, and a badly shaped
    element's cofactors from the FP64 coordinates;
  - FP64 and F64X forms: |K| within a few units of rounding of the products det B is
    formed from (relative error <= 64 u P / |det B|, P the sum of the absolute values
    of its terms, u = 2^-53 for FP64, 2^-46 for F64X's double-float): no computation of
    det B in that arithmetic from rounded edges does better;
  - the FP32 form also against the FP64 oracle through the usual gates (the oracle's
    own error is of the conditioning-bound size, within the FP32 tolerance).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import PARITY_LOG, check_values, exact_p1_matrices, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu

FLAT = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10]


def det_conditioning(q, me):
    """Per element: P / |det B| in exact arithmetic, P = sum of |terms| of det B."""
    d = q.shape[0]
    out = []
    for k in range(me.shape[1]):
        X = [[Fraction(float(q[c, v])) for c in range(d)] for v in me[:, k]]
        E = [[X[i + 1][c] - X[0][c] for c in range(d)] for i in range(d)]
        det, P = Fraction(0), Fraction(0)
        for perm in itertools.permutations(range(d)):
            inv = sum(1 for i in range(d) for j in range(i + 1, d) if perm[i] > perm[j])
            t = Fraction(1)
            for i in range(d):
                t *= E[i][perm[i]]
            det += -t if inv % 2 else t
            P += abs(t)
        out.append(float(P / abs(det)))
    return np.array(out)


def entries(res, ex, which):
    rows = np.repeat(np.arange(res["n"]), np.diff(res["row_ptr"]))
    return np.array([float(ex[(int(r), int(c))][which]) for r, c in zip(rows, res["col_idx"])]), rows


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("center", [None, (1000.0, -2000.0, 3000.5)])
def test_badly_shaped_elements(d, center):
    fe = fe_or_skip()
    m = meshgen.badly_shaped_mesh(d, FLAT, seed=40 + d, center=None if center is None else center[:d])
    kappa = det_conditioning(m.q, m.me)
    assert kappa.max() > 1e9  # the family reaches det B / P below 1e-9
    ex = exact_p1_matrices(m.q, m.me)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me)
    rm = oracle.assemble(oracle.MASS, m.q, m.me)
    rs = oracle.assemble(oracle.STIFF, m.q, m.me)
    m_ex, rows = entries(rm, ex, 1)
    s_ex, _ = entries(rs, ex, 0)
    k_row = kappa[rows // (d + 1)]  # conditioning of the element of each entry (isolated elements)
    where = "far from the origin" if center else "near the origin"
    unit = {fe.F64: 2.0 ** -53, fe.F64X: 2.0 ** -46}
    for prec in (fe.F64, fe.F32, fe.F64X):
        mass = fe.fe_assemble_mass(p, q, prec=prec).double().cpu().numpy()
        stiff = fe.fe_assemble_stiff(p, q, prec=prec).double().cpu().numpy()
        assert p.status() == (0, -1)
        rel_k = np.abs(mass - m_ex) / np.abs(m_ex)
        norm_s = np.abs(stiff - s_ex) / np.maximum(np.abs(s_ex), rs["scale"])
        key = f"{d}D badly shaped elements, {where}, vs exact [{['FP64', 'FP32', 'F64X'][prec]}]"
        PARITY_LOG[key] = dict(norm=float(norm_s.max()), comp=float(rel_k.max()), comp_res=float(rel_k.max()),
                               plain=float(rel_k.max()), n_unres=0, n=int(mass.size), cases=1)
        if prec == fe.F32:
            assert rel_k.max() <= 1e-6, rel_k.max()
            assert norm_s.max() <= 1e-5, norm_s.max()
            check_values(mass, rm, prec, f"{d}D badly shaped elements, {where}: mass")
            check_values(stiff, rs, prec, f"{d}D badly shaped elements, {where}: stiffness")
        else:
            u = unit[prec]
            assert np.all(rel_k <= 64 * u * k_row), (prec, (rel_k / (u * k_row)).max())

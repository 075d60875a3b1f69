"""Shared test helpers: library loading, oracle comparison and error metrics."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def fe_or_skip():
    """The binding, with the library built; skips when no CUDA device is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_3301_gb300 import build_ext, fe
    build_ext.build()
    fe.lib()
    return fe


def to_cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# Per-form tolerance and unit roundoff (prec 0 = FP64, 1 = FP32, 2 = F64X; F64X is
# double-float arithmetic, about 47 significant bits, on coordinates taken relative to a
# reference vertex of the element chunk). RESOLVE = 16: a form's arithmetic errors in an
# entry stay within about 16 units of its roundoff of the entry's normwise scale.
TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}
UNIT = {0: 2.0 ** -53, 1: 2.0 ** -24, 2: 2.0 ** -46}
RESOLVE = 16.0
FORM_NAME = {0: "FP64", 1: "FP32", 2: "F64X"}

# label -> {measure: max}, collected over the session and printed by conftest
PARITY_LOG: dict = {}


def value_errors(got, ref_val, ref_scale, ref_abs, unit=0.0, tol=1.0, well=1e-3):
    """Per-nonzero error measures of computed values a against the oracle's sums b.

    N_ij is the sum of the contributions' normwise scales (the size their arithmetic
    rounds at), A_ij the sum of |contributions| (the condition scale of the sum).
    norm:     |a - b| / max(|b|, N_ij)
    comp:     |a - b| / max(|b|, A_ij), over every entry (0 / 0 = 0, x / 0 = inf);
    comp_res: the same over the resolved entries, A_ij >= RESOLVE (unit / tol) N_ij: below
              that the contributions cancel to less than the form's own rounding of each
              of them can resolve at the tolerance (no implementation in that arithmetic,
              the FP64 oracle included, meets it there), and those entries are held to
              the normwise measure instead;
    plain:    |a - b| / |b| over the entries with |b| >= well A_ij, b != 0.
    Returns the measures and the counts n_unres (unresolved entries) and n_plain."""
    a = np.asarray(got, dtype=np.float64)
    b = np.asarray(ref_val, dtype=np.float64)
    if a.size == 0:
        return dict(norm=0.0, comp=0.0, comp_res=0.0, plain=0.0, n_unres=0, n_plain=0)
    d = np.abs(a - b)
    ab = np.abs(b)

    def ratio(den, sel=None):
        if sel is not None:
            d_, den = d[sel], den[sel]
        else:
            d_ = d
        if d_.size == 0:
            return 0.0
        pos = den > 0
        r = np.where(pos, d_ / np.where(pos, den, 1.0), np.where(d_ > 0, np.inf, 0.0))
        return float(np.max(r))

    res = ref_abs >= RESOLVE * (unit / tol) * ref_scale
    wsel = (ab >= well * ref_abs) & (ab > 0)
    plain = float(np.max(d[wsel] / ab[wsel])) if wsel.any() else 0.0
    dn = np.maximum(ab, ref_scale)
    dc = np.maximum(ab, ref_abs)
    return dict(norm=ratio(dn), comp=ratio(dc), comp_res=ratio(dc, res), plain=plain,
                n_unres=int((~res).sum()), n_plain=int(wsel.sum()))


def check_values(got, ref, prec, label, sl=slice(None)):
    """Gate computed values against an oracle result dict (entries sl of it), after
    logging the measures of value_errors under ``label``: the normwise error over every
    entry and the error against the sum of |contributions| over the resolved entries,
    both within the form's tolerance."""
    tol = TOL[prec]
    e = value_errors(got, ref["val"][sl], ref["scale"][sl], ref["abssum"][sl], UNIT[prec], tol)
    key = f"{label} [{FORM_NAME.get(prec, prec)}]"
    log = PARITY_LOG.setdefault(key, dict(norm=0.0, comp=0.0, comp_res=0.0, plain=0.0, n_unres=0,
                                          n_plain=0, n=0, cases=0))
    for k in ("norm", "comp", "comp_res", "plain"):
        log[k] = max(log[k], e[k])
    log["n_unres"] += e["n_unres"]
    log["n_plain"] += e["n_plain"]
    log["n"] += int(np.asarray(got).size)
    log["cases"] += 1
    assert e["norm"] <= tol, (label, FORM_NAME[prec], "normwise", e["norm"], tol)
    assert e["comp_res"] <= tol, (label, FORM_NAME[prec], "sum of |contributions|", e["comp_res"], tol)
    return e


def normalised_error(got, ref_val, ref_scale):
    """max over entries of |got - ref| / max(|ref|, scale): relative error per nonzero,
    with cancelling sums measured against the size of their contributions."""
    got = np.asarray(got, dtype=np.float64)
    den = np.maximum(np.abs(ref_val), ref_scale)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(got - ref_val) / den)) if got.size else 0.0


def assert_pattern_equal(p, ref, stream=None):
    rp, ci = p.csr(stream)
    np.testing.assert_array_equal(rp.cpu().numpy().astype(np.int64), ref["row_ptr"])
    np.testing.assert_array_equal(ci.cpu().numpy(), ref["col_idx"])


def sub_mesh_rows(me, rows_vertices, nq):
    """Elements that touch any of the given vertices (their rows are then complete)."""
    mark = np.zeros(nq, dtype=bool)
    mark[rows_vertices] = True
    keep = mark[me].any(axis=0)
    return np.nonzero(keep)[0]


def exact_p1_matrices(q, me):
    """Stiffness and mass entries of a P1 mesh in exact rational arithmetic: the coordinates
    are taken as the exact rationals the doubles are, c_a the rows of adj(B) (c_0 = -sum),
    stiffness |K| g_a.g_b = c_a.c_b / (d! |det B|), mass |det B| (1 + delta) / (d+2)!.
    Returns {(i, j): [stiffness, mass, sum |stiffness contributions|]}."""
    d = q.shape[0]
    out = {}
    for k in range(me.shape[1]):
        v = [int(x) for x in me[:, k]]
        X = [[Fraction(float(q[c, x])) for c in range(d)] for x in v]
        B = [[X[i + 1][c] - X[0][c] for i in range(d)] for c in range(d)]  # column i = edge i
        if d == 2:
            det = B[0][0] * B[1][1] - B[0][1] * B[1][0]
            adj = [[B[1][1], -B[0][1]], [-B[1][0], B[0][0]]]           # adj(B)
        else:
            det = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1])
                   - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0])
                   + B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]))
            adj = [[(B[(j + 1) % 3][(i + 1) % 3] * B[(j + 2) % 3][(i + 2) % 3]
                     - B[(j + 1) % 3][(i + 2) % 3] * B[(j + 2) % 3][(i + 1) % 3]) for j in range(3)]
                   for i in range(3)]
        c = [[-sum(adj[i][j] for i in range(d)) for j in range(d)]] + [adj[i] for i in range(d)]
        fd, f2 = math.factorial(d), math.factorial(d + 2)
        for a in range(d + 1):
            for b in range(d + 1):
                s = sum(c[a][j] * c[b][j] for j in range(d)) / (fd * abs(det))
                mval = abs(det) * (2 if a == b else 1) / f2
                e = out.setdefault((v[a], v[b]), [Fraction(0), Fraction(0), Fraction(0)])
                e[0] += s
                e[1] += mval
                e[2] += abs(s)
    return out

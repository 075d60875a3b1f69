"""Shared test helpers: library loading, oracle comparison and error metrics."""
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

"""Python access to the FP64 oracle (fe_oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``. The library's GPU path never imports it.

``build()`` compiles fe_oracle.c with the host C compiler into ``oracle/_build``.
The assembly arithmetic is in fe_oracle.c; the functions here convert arguments,
except ``pk_multi_indices``, ``_pk_basis`` and ``pk_mass_table``, which compute the
P_k node order and the exact-rational P_k mass table (App. D) in Python with
Fractions before the C assembly uses it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

MASS, WMASS, STIFF, ELAS = 0, 1, 2, 3
COEF_NONE, COEF_SCALAR, COEF_P0, COEF_P1 = 0, 1, 2, 3
ERRORS = {1: "argument", 2: "index", 3: "degenerate", 4: "out of memory"}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no vectorisation flags; with OpenMP where the
    compiler has it, for the threaded timing runs) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:3] + ["-fopenmp"] + base[3:], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
        lib.orc_magic.argtypes = [I32, P, D]
        lib.orc_magic.restype = D
        lib.orc_simplex.argtypes = [I32, P, P, P, P]
        lib.orc_element.argtypes = [I32, I32, P, P, P, P, P]
        lib.orc_assemble.argtypes = [I32, I32, I64, I64, P, P, I32, P, I32, P,
                                     P, P, P, P, P, P, P, P]
        lib.orc_stiff_loss.argtypes = [I32, I64, I64, P, P, P, P, P, P, P, P, P]
        lib.orc_facet.argtypes = [I32, P, P]
        lib.orc_assemble_boundary.argtypes = [I32, I32, I64, I64, P, P, I32, P, P, P, P, P, P, P, P, P]
        lib.orc_assemble_general.argtypes = [I32, I64, I64, P, P, I32, P, P, P, P, P, P, P, P, P]
        lib.orc_assemble_table.argtypes = [I32, I64, I64, I32, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_pattern.argtypes = [I32, I32, I64, I64, P, P, P, P, P]
        lib.orc_free.argtypes = [P]
        lib.orc_set_threads.argtypes = [I32]
        lib.orc_openmp.restype = I32
        lib.orc_slot_map.argtypes = [I32, I32, I64, I64, P, P, P, P, P]
        lib.orc_reassemble.argtypes = [I32, I32, I64, I64, P, P, I32, P, I32, P, I64, P, P, P, P]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, bad_id=-1):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}), id {bad_id}")
        self.code, self.bad_id = code, bad_id


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def magic(d: int, n, vol: float) -> float:
    n = np.ascontiguousarray(n, dtype=np.int32)
    return _load().orc_magic(d, _ptr(n), vol)


def simplex(X: np.ndarray):
    """(det B, |K|, G) for one simplex; X is (d+1, d); G is (d+1, d), row a = grad lambda_a."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    d = X.shape[1]
    det, vol = C.c_double(), C.c_double()
    G = np.zeros((d + 1, d))
    rc = _load().orc_simplex(d, _ptr(X), C.byref(det), C.byref(vol), _ptr(G))
    if rc:
        raise OracleError(rc)
    return det.value, vol.value, G


def element(kind: int, X: np.ndarray, cv1=None, cv2=None):
    """Local matrix (nl, nl) with E[i, j] = local entry (i, j), and its condition scale."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    d = X.shape[1]
    nl = (d + 1) * (d if kind == ELAS else 1)
    E = np.zeros(nl * nl)
    S = np.zeros(nl * nl)
    c1 = None if cv1 is None else np.ascontiguousarray(np.broadcast_to(cv1, (d + 1,)), dtype=np.float64)
    c2 = None if cv2 is None else np.ascontiguousarray(np.broadcast_to(cv2, (d + 1,)), dtype=np.float64)
    rc = _load().orc_element(kind, d, _ptr(X), _ptr(c1), _ptr(c2), _ptr(E), _ptr(S))
    if rc:
        raise OracleError(rc)
    # storage is column-wise: E[j*nl + i] holds local entry (i, j)
    return E.reshape(nl, nl).T.copy(), S.reshape(nl, nl).T.copy()


def _csr_result(lib, n, nnz, rp, ci, va, sc, sa) -> dict:
    """The malloc'ed CSR arrays of an oracle assembly as numpy arrays (freed after copying)."""

    def take(p, ctype, count, dtype):
        arr = np.ctypeslib.as_array(C.cast(p, C.POINTER(ctype)), shape=(max(count, 1),))[:count]
        out = np.array(arr, dtype=dtype)
        lib.orc_free(p)
        return out

    N, NNZ = n.value, nnz.value
    return dict(n=N, nnz=NNZ,
                row_ptr=take(rp, C.c_int64, N + 1, np.int64),
                col_idx=take(ci, C.c_int32, NNZ, np.int32),
                val=take(va, C.c_double, NNZ, np.float64),
                scale=take(sc, C.c_double, NNZ, np.float64),
                abssum=take(sa, C.c_double, NNZ, np.float64))


def _coef(c):
    """(kind, array) for a coefficient given as None, a number, or a per-element/vertex array."""
    if c is None:
        return COEF_NONE, None
    if np.isscalar(c):
        return COEF_SCALAR, np.array([float(c)])
    kind, arr = c
    return kind, np.ascontiguousarray(arr, dtype=np.float64)


def assemble(kind: int, q: np.ndarray, me: np.ndarray, c1=None, c2=None) -> dict:
    """Assemble the global matrix. c1/c2: None, a number, or (COEF_P0|COEF_P1, array).

    Returns dict(n, nnz, row_ptr int64, col_idx int32, val float64, scale float64,
    abssum float64): per entry the sum, the sum of its contributions' normwise condition
    scales, and the sum of their absolute values.
    """
    q = np.ascontiguousarray(q, dtype=np.float64)
    me = np.ascontiguousarray(me, dtype=np.int32)
    d, nq = q.shape
    nme = me.shape[1]
    k1, a1 = _coef(c1)
    k2, a2 = _coef(c2)
    n, nnz, bad = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ci, va, sc, sa = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_assemble(kind, d, nq, nme, _ptr(q), _ptr(me), k1, _ptr(a1), k2, _ptr(a2),
                          C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(va),
                          C.byref(sc), C.byref(sa), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)

    return _csr_result(lib, n, nnz, rp, ci, va, sc, sa)


def pattern(me: np.ndarray, nq: int, m: int = 1) -> tuple:
    """(row_ptr int64, col_idx int32) of the assembled matrix's nonzero pattern alone,
    with m dofs per vertex, from the connectivity me ((d+1) x nme)."""
    me = np.ascontiguousarray(me, dtype=np.int32)
    d = me.shape[0] - 1
    nnz, bad = C.c_int64(), C.c_int64()
    rp, ci = C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_pattern(d, m, nq, me.shape[1], _ptr(me), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)
    n, NNZ = m * nq, nnz.value
    row_ptr = np.array(np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_int64)), shape=(n + 1,)), dtype=np.int64)
    col_idx = np.array(np.ctypeslib.as_array(C.cast(ci, C.POINTER(C.c_int32)), shape=(max(NNZ, 1),))[:NNZ],
                       dtype=np.int32)
    lib.orc_free(rp)
    lib.orc_free(ci)
    return row_ptr, col_idx


def set_threads(n: int) -> int:
    """Threads of the oracle's element loops and sorts (1 by default; without OpenMP in
    the build always 1). Results do not depend on it. Returns the count in effect."""
    lib = _load()
    n = max(1, int(n)) if lib.orc_openmp() else 1
    lib.orc_set_threads(n)
    return n


def slot_map(me: np.ndarray, nq: int, m: int = 1) -> tuple:
    """(nnz_ptr, nnz2slot) int64: the element slots k ns + slot of each nonzero, in the
    order orc_assemble sums them (see fe_oracle.c, orc_slot_map)."""
    me = np.ascontiguousarray(me, dtype=np.int32)
    d = me.shape[0] - 1
    nnz, bad = C.c_int64(), C.c_int64()
    pp, ps = C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_slot_map(d, m, nq, me.shape[1], _ptr(me), C.byref(nnz), C.byref(pp), C.byref(ps), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)
    nt = me.shape[1] * (m * (d + 1)) ** 2
    ptr = np.array(np.ctypeslib.as_array(C.cast(pp, C.POINTER(C.c_int64)), shape=(nnz.value + 1,)), dtype=np.int64)
    n2s = np.array(np.ctypeslib.as_array(C.cast(ps, C.POINTER(C.c_int64)), shape=(max(nt, 1),))[:nt], dtype=np.int64)
    lib.orc_free(pp)
    lib.orc_free(ps)
    return ptr, n2s


def reassemble(kind: int, q: np.ndarray, me: np.ndarray, nnz_ptr: np.ndarray, nnz2slot: np.ndarray,
               c1=None, c2=None) -> np.ndarray:
    """Fixed-pattern reassembly: the values of assemble(kind, q, me, c1, c2) from the slot
    map of slot_map(me, nq), bit for bit."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    me = np.ascontiguousarray(me, dtype=np.int32)
    d, nq = q.shape
    k1, a1 = _coef(c1)
    k2, a2 = _coef(c2)
    nnz = len(nnz_ptr) - 1
    val = np.empty(nnz)
    bad = C.c_int64()
    ptr = np.ascontiguousarray(nnz_ptr, dtype=np.int64)
    n2s = np.ascontiguousarray(nnz2slot, dtype=np.int64)
    rc = _load().orc_reassemble(kind, d, nq, me.shape[1], _ptr(q), _ptr(me), k1, _ptr(a1), k2, _ptr(a2), nnz,
                                _ptr(ptr), _ptr(n2s), _ptr(val), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)
    return val


def facet_measure(X: np.ndarray) -> float:
    """Measure of a (d-1)-simplex in d-space; X is (d, d): one vertex per row."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    meas = C.c_double()
    rc = _load().orc_facet(X.shape[1], _ptr(X), C.byref(meas))
    if rc:
        raise OracleError(rc)
    return meas.value


def assemble_boundary(kind: int, q: np.ndarray, facets: np.ndarray, c1=None) -> dict:
    """Boundary (facet) mass / weighted mass; same result dict as assemble()."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    fa = np.ascontiguousarray(facets, dtype=np.int32)
    d, nq = q.shape
    k1, a1 = _coef(c1)
    n, nnz, bad = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ci, va, sc, sa = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_assemble_boundary(kind, d, nq, fa.shape[1], _ptr(q), _ptr(fa), k1, _ptr(a1),
                                   C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(va),
                                   C.byref(sc), C.byref(sa), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)

    return _csr_result(lib, n, nnz, rp, ci, va, sc, sa)


def assemble_general(q: np.ndarray, me: np.ndarray, coef: np.ndarray, kind: int) -> dict:
    """General operator of Eq. EDP. coef: records of the nc = d*d + 2d + 1 values A
    (row-major), b, c, a0: (nc,) for COEF_SCALAR, (nme, nc) for COEF_P0, (nq, nc) for
    COEF_P1. Same result dict as assemble()."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    me = np.ascontiguousarray(me, dtype=np.int32)
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    d, nq = q.shape
    n, nnz, bad = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ci, va, sc, sa = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_assemble_general(d, nq, me.shape[1], _ptr(q), _ptr(me), kind,
                                  _ptr(cf), C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(va),
                                  C.byref(sc), C.byref(sa), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)

    return _csr_result(lib, n, nnz, rp, ci, va, sc, sa)


def pk_multi_indices(d: int, k: int) -> list:
    """The P_k nodes of a d-simplex as multi-indices alpha (|alpha| = k, d+1 entries), in
    the local node order: the d+1 vertices k e_0, ..., k e_d first, then every other alpha
    in lexicographically decreasing order."""
    verts = [tuple(k if i == j else 0 for i in range(d + 1)) for j in range(d + 1)]
    rest = sorted((a for a in product(range(k + 1), repeat=d + 1) if sum(a) == k and a not in verts),
                  reverse=True)
    return verts + rest


def _pk_basis(alpha, k):
    """phi_alpha of Eq. Pk:functions as {mu: coefficient} over barycentric monomials."""
    poly = {tuple(0 for _ in alpha): Fraction(1)}
    for l, al in enumerate(alpha):
        for j in range(al):  # times (k lambda_l - j) / (j + 1)
            nxt = {}
            for mu, c in poly.items():
                up = list(mu)
                up[l] += 1
                up = tuple(up)
                nxt[up] = nxt.get(up, 0) + c * Fraction(k, j + 1)
                nxt[mu] = nxt.get(mu, 0) - c * Fraction(j, j + 1)
            poly = {m: c for m, c in nxt.items() if c != 0}
    return poly


def pk_mass_table(d: int, k: int) -> list:
    """Exact (integral of phi_alpha phi_beta) / |K| for all node pairs (list of rows of
    Fractions, local node order), by the magic formula (Eq. MagicFormula) applied to the
    monomial expansion of the basis functions."""
    al = pk_multi_indices(d, k)
    basis = [_pk_basis(a, k) for a in al]

    def magic(n):  # integral of prod lambda^n over K, divided by |K|
        num = factorial(d)
        for x in n:
            num *= factorial(x)
        return Fraction(num, factorial(d + sum(n)))

    tab = []
    for pa in basis:
        row = []
        for pb in basis:
            s = Fraction(0)
            for mu, ca in pa.items():
                for nu, cb in pb.items():
                    s += ca * cb * magic([x + y for x, y in zip(mu, nu)])
            row.append(s)
        tab.append(row)
    return tab


def assemble_pk_mass(q: np.ndarray, me: np.ndarray, k: int) -> dict:
    """P_k mass matrix (App. D, Algorithm 15) of a P_k mesh whose rows of me follow
    pk_multi_indices. Same result dict as assemble()."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    me = np.ascontiguousarray(me, dtype=np.int32)
    d, nq = q.shape
    tab = np.array([[float(x) for x in row] for row in pk_mass_table(d, k)])
    ndfe = tab.shape[0]
    assert me.shape[0] == ndfe
    flat = np.ascontiguousarray(tab.T)  # flat[b * ndfe + a] = entry (a, b)
    n, nnz, bad = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ci, va, sc, sa = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    lib = _load()
    rc = lib.orc_assemble_table(d, nq, me.shape[1], ndfe, _ptr(q), _ptr(me), _ptr(flat), C.byref(n),
                                C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(va), C.byref(sc),
                                C.byref(sa), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)

    return _csr_result(lib, n, nnz, rp, ci, va, sc, sa)


def stiff_loss(q, me, w, u, v, grads: bool = True):
    """(L, dL/dw, dL/dq) for L = u^T K(w) v, K the stiffness matrix; w per element or None."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    me = np.ascontiguousarray(me, dtype=np.int32)
    d, nq = q.shape
    nme = me.shape[1]
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    L, bad = C.c_double(), C.c_int64()
    dw = np.zeros(nme) if grads else None
    dq = np.zeros((d, nq)) if grads else None
    rc = _load().orc_stiff_loss(d, nq, nme, _ptr(q), _ptr(me), _ptr(w), _ptr(u), _ptr(v),
                                C.byref(L), _ptr(dw), _ptr(dq), C.byref(bad))
    if rc:
        raise OracleError(rc, bad.value)
    return L.value, dw, dq


def to_dense(res: dict) -> np.ndarray:
    """Dense copy of an oracle CSR result (small cases only)."""
    n = res["n"]
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(res["row_ptr"]))
    A[rows, res["col_idx"]] = res["val"]
    return A

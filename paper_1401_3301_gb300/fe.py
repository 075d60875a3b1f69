"""Thin Python binding of the C ABI in include/fe.h (argument marshalling only).

Every function has the name of the C entry point it calls and takes torch CUDA
tensors; all arithmetic happens in libfe_gb300.so. There is no CPU fallback: if
the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build_ext

F64, F32, F64X = 0, 1, 2
COEF_NONE, COEF_SCALAR, COEF_P0, COEF_P1, COEF_P0_INTERNAL = 0, 1, 2, 3, 4
REASM_CHUNKED, REASM_GATHER, REASM_ATOMIC = 0, 1, 2
PATTERN_KEEP_ORDER = 1
PATTERN_ENTITY_ORDER = 2
PATTERN_INTERLEAVED = 4


def PATTERN_CHUNK(c: int) -> int:
    """Pattern flag: elements per chunk of the chunked reassembly (32..4096)."""
    return int(c) << 8
ERRORS = {1: "FE_ERR_ARG", 2: "FE_ERR_INDEX", 3: "FE_ERR_DEGENERATE", 4: "FE_ERR_OVERFLOW",
          5: "FE_ERR_CUDA", 6: "FE_ERR_TIMEOUT", 7: "FE_ERR_NOMEM", 8: "FE_ERR_SCRATCH_LIMIT", 9: "FE_ERR_BOUNDS"}

_lib = None


class FEError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        super().__init__(f"{ERRORS.get(code, code)}{': ' + detail if detail else ''}")
        self.code = code


def lib() -> C.CDLL:
    """The loaded libfe_gb300.so (raises if it has not been built). With the environment
    variable FE_GB300_CHECKED=1 the bounds-checked build is loaded instead."""
    global _lib
    if _lib is None:
        path = build_ext.LIB_CHECKED if os.environ.get("FE_GB300_CHECKED") == "1" else build_ext.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libfe_gb300.so is missing ({path}); build it with "
                               "paper_1401_3301_gb300.build_ext.build()")
        L = C.CDLL(path)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        L.fe_pattern.argtypes = [P, I32, I32, P, P]
        L.fe_pattern_copy_csr.argtypes = [P, P, P, P]
        L.fe_pattern_copy_slot_map.argtypes = [P, P, P, P, P, P]
        L.fe_pattern_dims.argtypes = [P, P, P, P, P, P, P]
        L.fe_pattern_set_strategy.argtypes = [P, I32]
        L.fe_pattern_memory.argtypes = [P, P]
        L.fe_pattern_plan_info.argtypes = [P, P, P, P, P, P, P, P, P]
        L.fe_pattern_plan_record.argtypes = [P, I64, P, P]
        L.fe_pattern_destroy.argtypes = [P]
        L.fe_status.argtypes = [P, P, P, P]
        L.fe_assemble_mass.argtypes = [P, P, I32, P, P]
        L.fe_assemble_wmass.argtypes = [P, P, P, I32, I32, P, P]
        L.fe_assemble_stiff.argtypes = [P, P, P, I32, I32, P, P]
        L.fe_assemble_wmass_stiff.argtypes = [P, P, P, I32, I32, P, P, P]
        L.fe_pattern_set_persistent.argtypes = [P, I32]
        L.fe_assemble_elas.argtypes = [P, P, P, I32, P, I32, I32, P, P]
        L.fe_assemble_general.argtypes = [P, P, P, I32, I32, P, P]
        L.fe_pk_pattern.argtypes = [P, I32, I32, P, P]
        L.fe_pk_mass_table.argtypes = [I32, I32, P]
        L.fe_morton_vertex_order.argtypes = [I32, I64, P, P, P]
        L.fe_assemble_stiff_host.argtypes = [P, P, P, I32, I32, P, P]
        L.fe_selftest_wait_timeout.argtypes = [P, P]
        L.fe_apply_vertex_order.argtypes = [I32, I64, I64, I32, P, P, P, P, P, P]
        L.fe_assemble_stiff_backward.argtypes = [P, P, P, I32, P, P, P, P, P, I32, P]
        L.fe_assemble_stiff_noalloc.argtypes = [P, P, P, I32, I32, P, P]
        L.fe_assemble_stiff_vjp.argtypes = [P, P, P, I32, P, P, P, I32, P]
        L.fe_batch_pattern.argtypes = [P, I32, I32, I32, P, P]
        L.fe_boundary_pattern.argtypes = [P, I32, P, P]
        L.fe_pattern_set_threads.argtypes = [P, I32]
        L.fe_batch_offsets.argtypes = [P, P, P, P]
        L.fe_batch_count.argtypes = [P, P]
        L.fe_batch_gather_q.argtypes = [P, P, P, P]
        L.fe_profile.argtypes = [P, I32]
        L.fe_profile_read.argtypes = [P, I32, P, P, P, P]
        L.fe_version.restype = C.c_char_p
        L.fe_last_cuda_error.restype = C.c_char_p
        for name in ("fe_pattern", "fe_pattern_copy_csr", "fe_pattern_copy_slot_map", "fe_pattern_dims",
                     "fe_pattern_set_strategy", "fe_pattern_memory", "fe_pattern_plan_info",
                     "fe_pattern_destroy", "fe_pattern_plan_record", "fe_status", "fe_assemble_mass",
                     "fe_assemble_wmass",
                     "fe_assemble_stiff", "fe_assemble_elas", "fe_assemble_stiff_backward",
                     "fe_profile", "fe_profile_read", "fe_assemble_stiff_noalloc",
                     "fe_assemble_stiff_vjp", "fe_batch_pattern", "fe_batch_offsets",
                     "fe_batch_count", "fe_batch_gather_q", "fe_pattern_set_threads",
                     "fe_boundary_pattern", "fe_assemble_general", "fe_pk_pattern", "fe_pk_mass_table",
                     "fe_morton_vertex_order", "fe_apply_vertex_order", "fe_assemble_stiff_host",
                     "fe_selftest_wait_timeout", "fe_assemble_wmass_stiff", "fe_pattern_set_persistent"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise FEError(rc, lib().fe_last_cuda_error().decode() if rc in (5, 7) else "")


def _stream(stream) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor | None, dtype=None, name="tensor") -> C.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class _Mesh(C.Structure):
    _fields_ = [("d", C.c_int32), ("nq", C.c_int64), ("nme", C.c_int64), ("q", C.c_void_p),
                ("me", C.c_void_p)]


def _vtype(prec: int):
    return torch.float32 if prec == F32 else torch.float64


class Pattern:
    """Owner of an fe_pattern_h handle."""

    def __init__(self, handle: C.c_void_p):
        self.handle = handle
        d, m = C.c_int32(), C.c_int32()
        nq, nme, n, nnz = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().fe_pattern_dims(handle, C.byref(d), C.byref(m), C.byref(nq), C.byref(nme),
                                     C.byref(n), C.byref(nnz)))
        self.d, self.m, self.nq, self.nme, self.n, self.nnz = (d.value, m.value, nq.value, nme.value,
                                                               n.value, nnz.value)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.handle is not None and _lib is not None:
            _lib.fe_pattern_destroy(self.handle)
        self.handle = None

    def csr(self, stream=None):
        """(row_ptr, col_idx): int32 CUDA tensors (copies)."""
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        _check(lib().fe_pattern_copy_csr(self.handle, _dev(rp), _dev(ci), _stream(stream)))
        return rp, ci

    def slot_map(self, stream=None):
        """(slot2nnz, nnz_slot_ptr, nnz2slot, order) of the scalar pattern (copies)."""
        S = (self.d + 1) ** 2
        s2n = torch.empty(self.nme * S, dtype=torch.int32, device="cuda")
        nsp = torch.empty(self.nnz // (self.m * self.m) + 1, dtype=torch.int32, device="cuda")
        n2s = torch.empty(self.nme * S, dtype=torch.int32, device="cuda")
        order = torch.empty(self.nme, dtype=torch.int32, device="cuda")
        _check(lib().fe_pattern_copy_slot_map(self.handle, _dev(s2n), _dev(nsp), _dev(n2s), _dev(order),
                                              _stream(stream)))
        return s2n, nsp, n2s, order

    def element_order(self, stream=None) -> torch.Tensor:
        order = torch.empty(self.nme, dtype=torch.int32, device="cuda")
        _check(lib().fe_pattern_copy_slot_map(self.handle, None, None, None, _dev(order), _stream(stream)))
        return order

    def set_strategy(self, strategy: int):
        _check(lib().fe_pattern_set_strategy(self.handle, strategy))

    def set_threads(self, threads: int):
        _check(lib().fe_pattern_set_threads(self.handle, threads))

    def set_persistent(self, persistent: bool):
        _check(lib().fe_pattern_set_persistent(self.handle, 1 if persistent else 0))

    def memory(self) -> int:
        b = C.c_int64()
        _check(lib().fe_pattern_memory(self.handle, C.byref(b)))
        return b.value

    def plan_info(self) -> dict:
        keys = ("chunk", "local_vertices", "local_edges", "partial_vertices", "partial_edges",
                "shared_vertices", "shared_edges", "plan_bytes")
        v = [C.c_int64() for _ in keys]
        _check(lib().fe_pattern_plan_info(self.handle, *[C.byref(x) for x in v]))
        return dict(zip(keys, (x.value for x in v)))

    def plan_record(self, c: int) -> tuple[int, int]:
        """(device address, bytes) of element chunk c's plan record (borrowed)."""
        ptr, nb = C.c_void_p(), C.c_int64()
        _check(lib().fe_pattern_plan_record(self.handle, c, C.byref(ptr), C.byref(nb)))
        return ptr.value, nb.value

    def profile(self, enable: bool = True):
        _check(lib().fe_profile(self.handle, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read (synchronises)."""
        n = 16
        names = C.create_string_buffer(32 * n)
        ms = (C.c_double * n)()
        launches = (C.c_int64 * n)()
        count = C.c_int32()
        _check(lib().fe_profile_read(self.handle, n, names, ms, launches, C.byref(count)))
        out = {}
        for k in range(min(count.value, n)):
            nm = names.raw[32 * k:32 * k + 32].split(b"\0")[0].decode()
            out[nm] = (ms[k], launches[k])
        return out

    def status(self, stream=None):
        """(code, element id) from the device status word; clears it."""
        code, eid = C.c_int32(), C.c_int64()
        _check(lib().fe_status(self.handle, _stream(stream), C.byref(code), C.byref(eid)))
        return code.value, eid.value

    def check(self, stream=None):
        code, eid = self.status(stream)
        if code:
            raise FEError(code, f"element {eid}")


def fe_pattern(q: torch.Tensor, me: torch.Tensor, m: int = 1, flags: int = 0, stream=None) -> Pattern:
    d = q.shape[0]
    mesh = _Mesh(d, q.shape[1], me.shape[1], _dev(q, torch.float64, "q").value,
                 _dev(me, torch.int32, "me").value)
    if me.shape[0] != d + 1:
        raise ValueError("me must be (d+1, nme)")
    h = C.c_void_p()
    _check(lib().fe_pattern(C.byref(mesh), m, flags, _stream(stream), C.byref(h)))
    return Pattern(h)


def _meshes(qs, mes):
    arr = (_Mesh * len(qs))()
    for b, (q, me) in enumerate(zip(qs, mes)):
        if me.shape[0] != q.shape[0] + 1:
            raise ValueError("me must be (d+1, nme)")
        arr[b] = _Mesh(q.shape[0], q.shape[1], me.shape[1], _dev(q, torch.float64, "q").value,
                       _dev(me, torch.int32, "me").value)
    return arr


def fe_boundary_pattern(q: torch.Tensor, facets: torch.Tensor, flags: int = 0, stream=None) -> Pattern:
    """Pattern of a mesh of boundary facets ((d-1)-simplices in d-space, d rows of vertices)."""
    d = q.shape[0]
    if facets.shape[0] != d:
        raise ValueError("facets must be (d, nfacets)")
    mesh = _Mesh(d, q.shape[1], facets.shape[1], _dev(q, torch.float64, "q").value,
                 _dev(facets, torch.int32, "facets").value)
    h = C.c_void_p()
    _check(lib().fe_boundary_pattern(C.byref(mesh), flags, _stream(stream), C.byref(h)))
    return Pattern(h)


def fe_pk_pattern(q: torch.Tensor, me: torch.Tensor, k: int, flags: int = 0, stream=None) -> Pattern:
    """Pattern of a P_k mesh (App. D): me has (d+k)!/(d! k!) rows in the node order of
    include/fe.h (vertices first); fe_assemble_mass then gives the P_k mass matrix."""
    d = q.shape[0]
    ndfe = 1
    for i in range(1, d + 1):
        ndfe = ndfe * (k + i) // i
    if me.dim() != 2 or me.shape[0] != ndfe:
        raise ValueError(f"me must be ({ndfe}, nme) for P{k} elements in {d}D")
    mesh = _Mesh(d, q.shape[1], me.shape[1], _dev(q, torch.float64, "q").value, _dev(me, torch.int32, "me").value)
    h = C.c_void_p()
    _check(lib().fe_pk_pattern(C.byref(mesh), k, flags, _stream(stream), C.byref(h)))
    return Pattern(h)


def fe_morton_vertex_order(q: torch.Tensor, stream=None) -> torch.Tensor:
    """order[i] = the vertex placed at position i along a Morton curve (int32, on q's device)."""
    d, nq = q.shape
    order = torch.empty(nq, dtype=torch.int32, device=q.device)
    _check(lib().fe_morton_vertex_order(d, nq, _dev(q, torch.float64, "q"), _dev(order, torch.int32, "order"),
                                        _stream(stream)))
    return order


def fe_apply_vertex_order(q: torch.Tensor, me: torch.Tensor, order: torch.Tensor, stream=None):
    """(q_out, me_out): the mesh with vertex order[i] renumbered i."""
    d, nq = q.shape
    q_out = torch.empty_like(q)
    me_out = torch.empty_like(me)
    _check(lib().fe_apply_vertex_order(d, nq, me.shape[1], me.shape[0], _dev(q, torch.float64, "q"),
                                       _dev(me, torch.int32, "me"), _dev(order, torch.int32, "order"),
                                       _dev(q_out, torch.float64, "q_out"), _dev(me_out, torch.int32, "me_out"),
                                       _stream(stream)))
    return q_out, me_out


def fe_pk_mass_table(d: int, k: int):
    """The constants C_{alpha,beta} of Eq. MatElemMassPk, (ndfe, ndfe) numpy float64."""
    import numpy as np
    n = 1
    for i in range(1, d + 1):
        n = n * (k + i) // i
    out = np.zeros((n, n))
    _check(lib().fe_pk_mass_table(d, k, out.ctypes.data_as(C.c_void_p)))
    return out


def fe_batch_pattern(qs: list, mes: list, m: int = 1, flags: int = 0, stream=None) -> Pattern:
    """Pattern of the disjoint union of several meshes (see include/fe.h)."""
    arr = _meshes(qs, mes)
    h = C.c_void_p()
    _check(lib().fe_batch_pattern(arr, len(qs), m, flags, _stream(stream), C.byref(h)))
    p = Pattern(h)
    p._batch_keep = (qs, mes)
    return p


def fe_batch_offsets(p: Pattern):
    """(vertex, element, nonzero) offsets of the meshes of a batch pattern, numpy int64."""
    import numpy as np
    cnt = C.c_int32()
    _check(lib().fe_batch_count(p.handle, C.byref(cnt)))
    n = cnt.value + 1
    vo, eo, no = (np.zeros(n, dtype=np.int64) for _ in range(3))
    _check(lib().fe_batch_offsets(p.handle, vo.ctypes.data_as(C.c_void_p), eo.ctypes.data_as(C.c_void_p),
                                  no.ctypes.data_as(C.c_void_p)))
    return vo, eo, no


def fe_batch_gather_q(p: Pattern, qs: list, mes: list, q_union: torch.Tensor, stream=None):
    arr = _meshes(qs, mes)
    _check(lib().fe_batch_gather_q(p.handle, arr, _dev(q_union, torch.float64, "q_union"), _stream(stream)))
    return q_union


def _out(p: Pattern, vals, prec):
    if vals is None:
        vals = torch.empty(p.nnz, dtype=_vtype(prec), device="cuda")
    return vals


def fe_assemble_mass(p: Pattern, q: torch.Tensor, prec: int = F64, vals=None, stream=None):
    vals = _out(p, vals, prec)
    _check(lib().fe_assemble_mass(p.handle, _dev(q, torch.float64, "q"), prec,
                                  _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_assemble_wmass(p: Pattern, q: torch.Tensor, w: torch.Tensor, w_kind: int = COEF_P1,
                      prec: int = F64, vals=None, stream=None):
    vals = _out(p, vals, prec)
    _check(lib().fe_assemble_wmass(p.handle, _dev(q, torch.float64, "q"), _dev(w, _vtype(prec), "w"),
                                   w_kind, prec, _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_assemble_stiff(p: Pattern, q: torch.Tensor, w: torch.Tensor | None = None,
                      w_kind: int | None = None, prec: int = F64, vals=None, stream=None):
    vals = _out(p, vals, prec)
    if w_kind is None:
        w_kind = COEF_NONE if w is None else COEF_P0
    _check(lib().fe_assemble_stiff(p.handle, _dev(q, torch.float64, "q"), _dev(w, _vtype(prec), "w"),
                                   w_kind, prec, _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_assemble_wmass_stiff(p: Pattern, q: torch.Tensor, w: torch.Tensor | None = None,
                            w_kind: int | None = None, prec: int = F64, vals_mass=None, vals_stiff=None,
                            stream=None):
    """(weighted mass, stiffness) with one per-element coefficient, in one pass (include/fe.h)."""
    vals_mass = _out(p, vals_mass, prec)
    vals_stiff = _out(p, vals_stiff, prec)
    if w_kind is None:
        w_kind = COEF_NONE if w is None else COEF_P0
    _check(lib().fe_assemble_wmass_stiff(p.handle, _dev(q, torch.float64, "q"), _dev(w, _vtype(prec), "w"), w_kind,
                                         prec, _dev(vals_mass, _vtype(prec), "vals_mass"),
                                         _dev(vals_stiff, _vtype(prec), "vals_stiff"), _stream(stream)))
    return vals_mass, vals_stiff


def fe_assemble_stiff_host(p: Pattern, q_host: torch.Tensor, vals_host: torch.Tensor, w_host=None,
                           prec: int = F64, stream=None):
    """fe_assemble_stiff from and to host tensors (pin them for overlap); asynchronous on
    `stream` like the device calls: synchronise before reading vals_host."""
    def host(t, dtype, name):
        if t is None:
            return None
        if t.device.type != "cpu" or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor of dtype {dtype}")
        return C.c_void_p(t.data_ptr())
    T = _vtype(prec)
    if vals_host.numel() != p.nnz:
        raise ValueError("vals_host must hold nnz values")
    if q_host.shape != (p.d, p.nq):
        raise ValueError("q_host must be (d, nq)")
    _check(lib().fe_assemble_stiff_host(p.handle, host(q_host, torch.float64, "q_host"), host(w_host, T, "w_host"),
                                        COEF_NONE if w_host is None else COEF_P0, prec,
                                        host(vals_host, T, "vals_host"), _stream(stream)))
    return vals_host


def fe_assemble_elas(p: Pattern, q: torch.Tensor, lam: torch.Tensor, lam_kind: int, mu: torch.Tensor,
                     mu_kind: int, prec: int = F64, vals=None, stream=None):
    vals = _out(p, vals, prec)
    _check(lib().fe_assemble_elas(p.handle, _dev(q, torch.float64, "q"), _dev(lam, _vtype(prec), "lam"),
                                  lam_kind, _dev(mu, _vtype(prec), "mu"), mu_kind, prec,
                                  _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_assemble_general(p: Pattern, q: torch.Tensor, coef: torch.Tensor, coef_kind: int, prec: int = F64,
                        vals=None, stream=None):
    """General operator of Eq. EDP; coef: records of nc = d*d + 2d + 1 values (A row-major,
    b, c, a0): one (COEF_SCALAR, shape (nc,)), one per element ((nme, nc), COEF_P0 /
    COEF_P0_INTERNAL) or one per vertex ((nq, nc), COEF_P1)."""
    vals = _out(p, vals, prec)
    _check(lib().fe_assemble_general(p.handle, _dev(q, torch.float64, "q"), _dev(coef, _vtype(prec), "coef"),
                                     coef_kind, prec, _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_assemble_stiff_backward(p: Pattern, q: torch.Tensor, w, w_kind: int, u: torch.Tensor,
                               v: torch.Tensor, L=None, dL_dw=None, dL_dq=None, prec: int = F64,
                               stream=None):
    T = _vtype(prec)
    _check(lib().fe_assemble_stiff_backward(
        p.handle, _dev(q, torch.float64, "q"), _dev(w, T, "w"), w_kind, _dev(u, T, "u"), _dev(v, T, "v"),
        _dev(L, T, "L"), _dev(dL_dw, T, "dL_dw"), _dev(dL_dq, T, "dL_dq"), prec, _stream(stream)))
    return L, dL_dw, dL_dq


def fe_assemble_stiff_vjp(p: Pattern, q: torch.Tensor, w, w_kind: int, grad_vals: torch.Tensor,
                          dL_dw=None, dL_dq=None, prec: int = F64, stream=None):
    T = _vtype(prec)
    _check(lib().fe_assemble_stiff_vjp(
        p.handle, _dev(q, torch.float64, "q"), _dev(w, T, "w"), w_kind, _dev(grad_vals, T, "grad_vals"),
        _dev(dL_dw, T, "dL_dw"), _dev(dL_dq, T, "dL_dq"), prec, _stream(stream)))
    return dL_dw, dL_dq


def fe_assemble_stiff_noalloc(p: Pattern, q: torch.Tensor, vals: torch.Tensor, w=None,
                              w_kind: int | None = None, prec: int = F64, stream=None):
    """Stiffness assembly that allocates no device memory (see include/fe.h): the
    caller passes the output buffer `vals` (nnz values of the form's precision)."""
    if w_kind is None:
        w_kind = COEF_NONE if w is None else COEF_P0
    _check(lib().fe_assemble_stiff_noalloc(p.handle, _dev(q, torch.float64, "q"), _dev(w, _vtype(prec), "w"),
                                           w_kind, prec, _dev(vals, _vtype(prec), "vals"), _stream(stream)))
    return vals


def fe_selftest_wait_timeout(stream=None) -> int:
    """Status code of a bounded wait that is made to run out (FE_ERR_TIMEOUT = 6 when the
    failure path works); see include/fe.h."""
    code = C.c_int32(-1)
    _check(lib().fe_selftest_wait_timeout(C.byref(code), _stream(stream)))
    return code.value


def fe_version() -> str:
    return lib().fe_version().decode()

"""Assemblies run twice by test_gpu_checked.py: once with the normal library and once,
in a child process with FE_GB300_CHECKED=1, with the bounds-checked build. Not a test
module itself (no test_ prefix)."""
import sys

import numpy as np


def run(fe) -> dict:
    """name -> numpy array of values, plus "status:<name>" -> (code, id) per assembly."""
    import torch
    from paper_1401_3301_gb300 import meshgen

    out = {}

    def cuda(a, dtype=None):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return (t.to(dtype) if dtype is not None else t).cuda()

    def record(name, p, vals):
        out[name] = vals.cpu().numpy().copy()
        out["status:" + name] = np.array(p.status(), dtype=np.int64)

    # 3D: several chunks, a ragged last chunk, both record layouts and two block sizes
    m3 = meshgen.kuhn_cube_mesh(13, seed=4)
    q3, me3 = cuda(m3.q), cuda(m3.me)
    w3 = cuda(meshgen.vertex_weights(4, m3.nq))
    e3 = cuda(meshgen.element_weights(4, m3.nme))
    for flags, threads in ((0, 256), (fe.PATTERN_ENTITY_ORDER | fe.PATTERN_CHUNK(256), 512)):
        p = fe.fe_pattern(q3, me3, flags=flags)
        p.set_threads(threads)
        tag = f"3d/{flags}/{threads}"
        for prec in (fe.F64, fe.F32, fe.F64X):
            record(f"{tag}/stiff/{prec}", p, fe.fe_assemble_stiff(p, q3, prec=prec))
        for prec in (fe.F64, fe.F32):
            T = torch.float64 if prec == fe.F64 else torch.float32
            record(f"{tag}/mass/{prec}", p, fe.fe_assemble_mass(p, q3, prec=prec))
            record(f"{tag}/wmass/{prec}", p, fe.fe_assemble_wmass(p, q3, w3.to(T), fe.COEF_P1, prec=prec))
            record(f"{tag}/stiffP0/{prec}", p, fe.fe_assemble_stiff(p, q3, e3.to(T), fe.COEF_P0, prec=prec))
    # 2D
    m2 = meshgen.square_mesh(37, seed=5)
    q2, me2 = cuda(m2.q), cuda(m2.me)
    p = fe.fe_pattern(q2, me2)
    for prec in (fe.F64, fe.F32):
        record(f"2d/stiff/{prec}", p, fe.fe_assemble_stiff(p, q2, prec=prec))
        record(f"2d/mass/{prec}", p, fe.fe_assemble_mass(p, q2, prec=prec))
    # the other kernels of the library, run under the checked build too
    pe = fe.fe_pattern(q3, me3, m=3)
    lam = torch.tensor([1.5], dtype=torch.float64, device="cuda")
    mu = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    record("3d/elas", pe, fe.fe_assemble_elas(pe, q3, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR))
    record("3d/elas/f64x", pe, fe.fe_assemble_elas(pe, q3, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR, prec=fe.F64X))
    record("3d/elas/f32", pe, fe.fe_assemble_elas(pe, q3, lam.float(), fe.COEF_SCALAR, mu.float(),
                                                  fe.COEF_SCALAR, prec=fe.F32))
    pb = fe.fe_boundary_pattern(q3, cuda(meshgen.boundary_facets(m3)))
    record("3d/boundary_mass", pb, fe.fe_assemble_mass(pb, q3))
    record("3d/boundary_wmass", pb, fe.fe_assemble_wmass(pb, q3, w3.float(), fe.COEF_P1, prec=fe.F32))
    record("3d/boundary_wmass/f64x", pb, fe.fe_assemble_wmass(pb, q3, w3, fe.COEF_P1, prec=fe.F64X))
    p = fe.fe_pattern(q3, me3)
    coef = cuda(meshgen.general_coefficients(4, 3, m3.nme))
    record("3d/general/p0", p, fe.fe_assemble_general(p, q3, coef, fe.COEF_P0))
    coef1 = cuda(meshgen.general_coefficients(5, 3, m3.nq))
    record("3d/general/p1", p, fe.fe_assemble_general(p, q3, coef1.float(), fe.COEF_P1, prec=fe.F32))
    record("3d/general/p0/f64x", p, fe.fe_assemble_general(p, q3, coef, fe.COEF_P0, prec=fe.F64X))
    record("3d/general/p1/f64x", p, fe.fe_assemble_general(p, q3, coef1, fe.COEF_P1, prec=fe.F64X))
    mk = meshgen.pk_mesh(3, 4, 2, seed=6)
    pk = fe.fe_pk_pattern(cuda(mk.q), cuda(mk.me), 2)
    record("3d/pk2_mass", pk, fe.fe_assemble_mass(pk, cuda(mk.q)))
    record("3d/pk2_mass/f64x", pk, fe.fe_assemble_mass(pk, cuda(mk.q), prec=fe.F64X))
    return out


class _DeviceInt16:
    """A borrowed device buffer seen as int16 through the CUDA array interface."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i2", "data": (ptr, False), "version": 3}


def corrupted(fe) -> dict:
    """Bounds-checked build only: corrupt chunk 1's plan record and assemble with every
    chunked kernel. The first word of the record is the local vertex of the chunk's first
    element corner: "duplicate" copies the second corner's into it, "range" makes it
    0xFFFF. For the tetrahedral patterns (chunk 1 full, 512 elements of 4 corners, so the
    vertex incidence lists start at word 2048) "inc" duplicates the second incidence code
    of the first list into the first. Each must report FE_ERR_BOUNDS for chunk 1 and skip it."""
    import torch
    from paper_1401_3301_gb300 import meshgen
    assert "bounds-checked" in fe.fe_version()  # the normal build would read out of bounds
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m3 = meshgen.kuhn_cube_mesh(13, seed=4)
    q3, me3 = cuda(m3.q), cuda(m3.me)
    mk = meshgen.pk_mesh(3, 6, 2, seed=6)
    qk = cuda(mk.q)
    lam = torch.tensor([1.5], dtype=torch.float64, device="cuda")
    coef = cuda(meshgen.general_coefficients(4, 3, m3.nme))
    cases = {
        "stiff/f64": (lambda: fe.fe_pattern(q3, me3), lambda p: fe.fe_assemble_stiff(p, q3)),
        "stiff/f32": (lambda: fe.fe_pattern(q3, me3), lambda p: fe.fe_assemble_stiff(p, q3, prec=fe.F32)),
        "stiff/f64x": (lambda: fe.fe_pattern(q3, me3), lambda p: fe.fe_assemble_stiff(p, q3, prec=fe.F64X)),
        "general": (lambda: fe.fe_pattern(q3, me3), lambda p: fe.fe_assemble_general(p, q3, coef, fe.COEF_P0)),
        "general/f64x": (lambda: fe.fe_pattern(q3, me3),
                         lambda p: fe.fe_assemble_general(p, q3, coef, fe.COEF_P0, prec=fe.F64X)),
        "elas": (lambda: fe.fe_pattern(q3, me3, m=3),
                 lambda p: fe.fe_assemble_elas(p, q3, lam, fe.COEF_SCALAR, lam, fe.COEF_SCALAR)),
        "elas/f64x": (lambda: fe.fe_pattern(q3, me3, m=3),
                      lambda p: fe.fe_assemble_elas(p, q3, lam, fe.COEF_SCALAR, lam, fe.COEF_SCALAR,
                                                    prec=fe.F64X)),
        "boundary": (lambda: fe.fe_boundary_pattern(q3, cuda(meshgen.boundary_facets(m3))),
                     lambda p: fe.fe_assemble_mass(p, q3)),
        "boundary/f64x": (lambda: fe.fe_boundary_pattern(q3, cuda(meshgen.boundary_facets(m3))),
                          lambda p: fe.fe_assemble_mass(p, q3, prec=fe.F64X)),
        "pk2": (lambda: fe.fe_pk_pattern(qk, cuda(mk.me), 2), lambda p: fe.fe_assemble_mass(p, qk)),
        "pk2/f64x": (lambda: fe.fe_pk_pattern(qk, cuda(mk.me), 2),
                     lambda p: fe.fe_assemble_mass(p, qk, prec=fe.F64X)),
    }
    tet = {"stiff/f64", "stiff/f32", "stiff/f64x", "general", "general/f64x", "elas", "elas/f64x"}
    out = {}
    for name, (make, assemble) in cases.items():
        for how in ("duplicate", "range", "inc") if name in tet else ("duplicate", "range"):
            p = make()
            assert p.nme > p.plan_info()["chunk"], name  # chunk 1 exists
            ptr, nbytes = p.plan_record(1)
            rec = torch.as_tensor(_DeviceInt16(ptr, nbytes // 2), device="cuda")
            if how == "duplicate":
                rec[0] = rec[1]
            elif how == "range":
                rec[0] = -1  # 0xFFFF
            else:
                assert p.plan_info()["chunk"] == 512, name
                rec[2048] = rec[2049]
            torch.cuda.synchronize()
            assemble(p)
            out[f"{name}/{how}"] = p.status()
            p.destroy()
    return out


def main(path: str) -> None:
    from paper_1401_3301_gb300 import fe
    out = run(fe)
    out["version"] = np.array(fe.fe_version())
    for name, st in corrupted(fe).items():
        out["corrupted:" + name] = np.array(st, dtype=np.int64)
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])

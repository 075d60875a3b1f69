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
    pb = fe.fe_boundary_pattern(q3, cuda(meshgen.boundary_facets(m3)))
    record("3d/boundary_mass", pb, fe.fe_assemble_mass(pb, q3))
    return out


def main(path: str) -> None:
    from paper_1401_3301_gb300 import fe
    out = run(fe)
    out["version"] = np.array(fe.fe_version())
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])

"""Autotuner: times a grid of chunk sizes / threads, caches the winner, and the
tuned pattern assembles the same matrix."""
import json

import numpy as np
import pytest

import oracle
from paper_1401_3301_gb300 import meshgen
from helpers import check_values, fe_or_skip, to_cuda

pytestmark = pytest.mark.gpu


def test_autotune_caches_and_tuned_pattern_is_correct(tmp_path, monkeypatch):
    fe = fe_or_skip()
    from paper_1401_3301_gb300 import tune
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("FE_TUNE_CACHE", str(cache))
    m = meshgen.kuhn_cube_mesh(10, seed=31)
    q, me = to_cuda(m.q), to_cuda(m.me)
    best = tune.autotune(q, me, chunks=(256, 512), threads=(128, 256), reps=3, deterministic_only=False)
    assert best["tried"] == 2 * 3 * 2 + 2 and best["ms"] > 0  # chunks x layouts x threads + 2 strategies
    stored = json.loads(cache.read_text())
    assert len(stored) == 1 and list(stored.values())[0]["ms"] == best["ms"]
    again = tune.autotune(q, me, chunks=(256, 512), threads=(128, 256), reps=3)
    assert again == best  # served from the cache
    p = tune.tuned_pattern(q, me, chunks=(256, 512), threads=(128, 256), reps=3)
    ref = oracle.assemble(oracle.STIFF, m.q, m.me)
    vals = fe.fe_assemble_stiff(p, q)
    check_values(vals.cpu().numpy(), ref, 0, "3D stiffness, tuned pattern")


def test_autotune_disabled_returns_defaults_untimed(tmp_path, monkeypatch):
    fe = fe_or_skip()
    from paper_1401_3301_gb300 import tune
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("FE_TUNE_CACHE", str(cache))
    monkeypatch.setenv("FE_AUTOTUNE", "0")
    m = meshgen.kuhn_cube_mesh(6, seed=32)
    q, me = to_cuda(m.q), to_cuda(m.me)
    assert tune.autotune(q, me) == tune.DEFAULT
    assert not cache.exists()  # nothing timed, nothing cached
    p = tune.tuned_pattern(q, me)
    assert p.plan_info()["chunk"] == fe.fe_pattern(q, me).plan_info()["chunk"]
    ref = oracle.assemble(oracle.STIFF, m.q, m.me)
    vals = fe.fe_assemble_stiff(p, q)
    check_values(vals.cpu().numpy(), ref, 0, "3D stiffness, tuned pattern")


@pytest.mark.parametrize("chunk,threads", [(256, 128), (768, 512), (1024, 256)])
def test_chunk_and_thread_variants_agree_with_oracle(chunk, threads):
    fe = fe_or_skip()
    m = meshgen.kuhn_cube_mesh(9, seed=32)
    q, me = to_cuda(m.q), to_cuda(m.me)
    p = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(chunk))
    p.set_threads(threads)
    assert p.plan_info()["chunk"] == chunk
    ref = oracle.assemble(oracle.STIFF, m.q, m.me)
    for prec in (0, 1):
        vals = fe.fe_assemble_stiff(p, q, prec=prec)
        check_values(vals.double().cpu().numpy(), ref, prec, "3D stiffness, tuned pattern")


def test_record_layouts_give_identical_values():
    # the count-ordered and the nonzero-ordered records change only which thread sums
    # which list; every sum keeps its element order, so the values agree bit for bit
    fe = fe_or_skip()
    import torch
    m = meshgen.kuhn_cube_mesh(9, seed=33)
    q, me = to_cuda(m.q), to_cuda(m.me)
    pa = fe.fe_pattern(q, me)
    pb = fe.fe_pattern(q, me, flags=fe.PATTERN_ENTITY_ORDER)
    w = to_cuda(meshgen.element_weights(3, m.nme))
    for prec in (fe.F64, fe.F32, fe.F64X):
        T = torch.float32 if prec == fe.F32 else torch.float64
        a = fe.fe_assemble_stiff(pa, q, w.to(T), fe.COEF_P0, prec=prec)
        b = fe.fe_assemble_stiff(pb, q, w.to(T), fe.COEF_P0, prec=prec)
        assert torch.equal(a, b), prec
    cf = to_cuda(meshgen.general_coefficients(4, 3, m.nme))
    assert torch.equal(fe.fe_assemble_general(pa, q, cf, fe.COEF_P0), fe.fe_assemble_general(pb, q, cf, fe.COEF_P0))
    ea, eb = fe.fe_pattern(q, me, m=3), fe.fe_pattern(q, me, m=3, flags=fe.PATTERN_ENTITY_ORDER)
    lam = torch.tensor([0.6], dtype=torch.float64, device="cuda")
    mu = torch.tensor([0.4], dtype=torch.float64, device="cuda")
    assert torch.equal(fe.fe_assemble_elas(ea, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR),
                       fe.fe_assemble_elas(eb, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR))

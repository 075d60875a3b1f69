"""Autotuner of the fixed-pattern reassembly.

For one mesh (or one batch of meshes) and operator it times the chunked kernel over a
grid of chunk sizes (elements per block, i.e. work per thread), the three layouts of the
chunk records (distinct vertices and edges by incidence count, in nonzero order, or
interleaved slots; a layout an operator or form does not take is skipped) and threads
per block, for the fused weighted mass + stiffness kernel also its launch shape
(persistent grid or one block per chunk), and optionally the two-pass gather and atomic
strategies, with CUDA events (median of `reps` calls after one warm-up). The winner is cached in a JSON file keyed by GPU name,
dimension, dofs per vertex, operator, precision and the element count's power of
two, so later meshes of the same class reuse it without timing. With the environment
variable FE_AUTOTUNE=0 nothing is timed and the library defaults are returned.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import build_ext, fe

CHUNKS = (224, 256, 384, 512, 768, 1024)
THREADS = (128, 256, 512)
PERSISTENT = (True, False)
LAYOUTS = (0, fe.PATTERN_ENTITY_ORDER, fe.PATTERN_INTERLEAVED)
_FORM = {fe.F64: "f64", fe.F32: "f32", fe.F64X: "f64x"}


def cache_path() -> str:
    return os.environ.get("FE_TUNE_CACHE", os.path.join(build_ext.BUILD, "tune.json"))


def enabled() -> bool:
    """False when FE_AUTOTUNE=0: autotune then returns the library defaults untimed."""
    return os.environ.get("FE_AUTOTUNE", "1") != "0"


# the configuration of a pattern built without flags (chunk 0: the library's default)
DEFAULT = {"strategy": "chunked", "chunk": 0, "layout": 0, "threads": 256, "persistent": True, "ms": None,
           "tried": 0}


def _key(d, m, kind, prec, nme) -> str:
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|d{d}|m{m}|{kind}|{_FORM[prec]}|2^{int(math.log2(max(nme, 1)))}"


def _call(p, q, kind, prec, w, w_kind, vals, vals2=None):
    if kind == "wmass_stiff":
        return fe.fe_assemble_wmass_stiff(p, q, w, w_kind, prec=prec, vals_mass=vals, vals_stiff=vals2)
    if kind == "stiff":
        return fe.fe_assemble_stiff(p, q, w, w_kind, prec=prec, vals=vals)
    if kind == "mass":
        return fe.fe_assemble_mass(p, q, prec=prec, vals=vals)
    if kind == "wmass":
        return fe.fe_assemble_wmass(p, q, w, w_kind, prec=prec, vals=vals)
    raise ValueError(f"unknown operator {kind}")


def _time(fn, reps: int) -> float:
    fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(q: torch.Tensor, me: torch.Tensor, kind: str = "stiff", prec: int = fe.F64, w=None,
             w_kind: int | None = None, reps: int = 10, chunks=CHUNKS, threads=THREADS, layouts=LAYOUTS,
             deterministic_only: bool = True, use_cache: bool = True, pattern=None, tag: str = "") -> dict:
    """Best {strategy, chunk, layout, threads, persistent, ms} for this mesh class, from the cache
    or by timing. pattern(flags) builds the pattern to tune (default fe_pattern(q, me, flags));
    tag distinguishes mesh classes in the cache key (e.g. batches). q is the coordinate array
    the assembly reads (for a batch, the union coordinates) and me sizes the element count."""
    if not enabled():
        return dict(DEFAULT)
    if w_kind is None:
        w_kind = fe.COEF_NONE if w is None else fe.COEF_P0
    d, nme = q.shape[0], me.shape[1]
    key = _key(d, 1, kind, prec, nme) + (f"|{tag}" if tag else "")
    if pattern is None:
        def pattern(flags):
            return fe.fe_pattern(q, me, flags=flags)
    path = cache_path()
    cache = _load(path)
    if use_cache and key in cache:
        return cache[key]
    T = torch.float32 if prec == fe.F32 else torch.float64
    # the launch shape applies to the FP64 / FP32 fused kernel only (F64X: one block per chunk)
    shapes = PERSISTENT if kind == "wmass_stiff" and prec != fe.F64X else (True,)
    results = []
    vals = vals2 = None
    if kind not in ("stiff", "mass", "wmass") or prec == fe.F64X:
        layouts = tuple(x for x in layouts if x != fe.PATTERN_INTERLEAVED)
    for c in chunks:
        for lay in layouts:
            p = pattern(fe.PATTERN_CHUNK(c) | lay)
            if vals is None:
                vals = torch.empty(p.nnz, dtype=T, device=q.device)
                vals2 = torch.empty(p.nnz, dtype=T, device=q.device) if kind == "wmass_stiff" else None
            for t in threads:
                p.set_threads(t)
                for per in shapes:
                    p.set_persistent(per)
                    try:
                        ms = _time(lambda: _call(p, q, kind, prec, w, w_kind, vals, vals2), reps)
                    except fe.FEError:  # chunk too large for one block's shared memory
                        continue
                    results.append({"strategy": "chunked", "chunk": c, "layout": lay, "threads": t,
                                    "persistent": per, "ms": ms})
            p.destroy()
    if not deterministic_only:
        p = pattern(0)
        for name, s in (("gather", fe.REASM_GATHER), ("atomic", fe.REASM_ATOMIC)):
            p.set_strategy(s)
            ms = _time(lambda: _call(p, q, kind, prec, w, w_kind, vals), reps)
            results.append({"strategy": name, "chunk": 0, "layout": 0, "threads": 256, "persistent": True,
                            "ms": ms})
        p.destroy()
    best = dict(min(results, key=lambda r: r["ms"]))
    best["tried"] = len(results)
    cache = _load(path)
    cache[key] = best
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best


def tuned_pattern(q: torch.Tensor, me: torch.Tensor, kind: str = "stiff", prec: int = fe.F64, pattern=None,
                  **kw) -> fe.Pattern:
    """A pattern built and configured with the autotuned chunk size, threads, launch shape
    and strategy (pattern: as for autotune)."""
    best = autotune(q, me, kind=kind, prec=prec, pattern=pattern, **kw)
    strategy = {"chunked": fe.REASM_CHUNKED, "gather": fe.REASM_GATHER, "atomic": fe.REASM_ATOMIC}[best["strategy"]]
    flags = (fe.PATTERN_CHUNK(best["chunk"]) if best["chunk"] else 0) | best.get("layout", 0)
    p = fe.fe_pattern(q, me, flags=flags) if pattern is None else pattern(flags)
    p.set_strategy(strategy)
    p.set_threads(best["threads"])
    p.set_persistent(best.get("persistent", True))
    return p

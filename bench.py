#!/usr/bin/env python
"""Benchmark: fixed-pattern reassembly of the 3D P1 stiffness matrix on GB300.

Workload: unit cube, N = 100 Kuhn 6-tetrahedron split (6,000,000 tets, 1,030,301
vertices, 15,210,901 nonzeros), interior vertices jittered by +-0.15 h, elements
randomly permuted (seeded). The sparsity pattern is built once, outside the timed
region; one step is one reassembly of the matrix values from the coordinates
(Algorithm 7 of Cuvelier-Japhet-Scarella followed by the value part of `sparse`).
Both precision forms are measured in the same run; --prec picks the one reported
as the headline value (FP64 by default, the precision of the paper).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
With N > 1 the script runs under torchrun, one process per GPU, each assembling
its own copy of the workload (independent replicas: the method needs no
exchange between meshes); value = tets of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D P1 stiffness Mtets/s and % HBM roofline, FP32 vs FP64 form, fixed pattern"
UNIT = "Mtets/s"
SM_COUNT = 152
FP64_PIPE_PER_SM_CLK = 2.0      # nominal FP64 issue rate per SM per clock on GB300
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["elem.cuh", "dfloat.cuh", "plan.cuh", "tma.cuh", "assemble_impl.cuh", "assemble_scalar.inc",
                  "assemble_f64.cu", "assemble_f32.cu", "assemble_f64x.cu"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="f64", choices=["f64", "f32"])
    ap.add_argument("--N", type=int, default=100, help="cells per cube side (default 100: 6M tets)")
    ap.add_argument("--strategy", default="chunked", choices=["chunked", "gather", "atomic"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help='per-form pattern configuration as JSON, e.g. \'{"f64": {"chunk": 384, "layout": 0, '
                         '"threads": 256}}\' (the dict a run prints in config.tuning); forms it names skip the '
                         'autotuner')
    ap.add_argument("--no-tune", action="store_true",
                    help="use the default pattern (chunk 512, count-ordered records, 256 threads) for every "
                         "form instead of the autotuned one")
    ap.add_argument("--cpu-sample", type=int, default=1_500_000, help="tets in the CPU-baseline sample")
    ap.add_argument("--workload", default="stiffness",
                    choices=["stiffness", "mass", "wmass", "elas", "2d", "batched", "diff", "general", "pk",
                             "boundary"],
                    help="stiffness (default, the headline); the others print one JSON line each "
                         "for the other configurations of the hot path")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_config(N, operator="stiffness"):
    nq, nme = (N + 1) ** 3, 6 * N ** 3
    return {"workload": f"3D P1 {operator}, fixed-pattern reassembly, Kuhn cube N={N} "
                        f"({nme:,} tets, {nq:,} vertices), jitter 0.15h, elements permuted",
            "mesh": "kuhn_cube", "N": N, "tets": nme, "vertices": nq}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured", float(pk.get("sm_max_mhz", 2070.0))
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", 2070.0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU baseline (oracle)
def host_cpu():
    """The host's CPU model (lscpu, else /proc/cpuinfo, else the machine type) and its
    logical CPU count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.split(":")[0].strip().lower() in ("model name", "cpu model", "hardware"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model or platform.machine(), "logical_cpus": os.cpu_count()}


def cpu_baseline(m, sample):
    import oracle
    oracle.build()
    S = min(sample, m.nme)
    me = np.ascontiguousarray(m.me[:, :S])
    t0 = time.perf_counter()
    oracle.assemble(oracle.STIFF, m.q, me)
    dt = time.perf_counter() - t0
    return {"value": S / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"first {S:,} of the {m.nme:,} randomly ordered tets of the same mesh "
                      f"(element loop + triplet sort-and-sum into CSR, FP64, one thread); {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1401_3301_gb300 import meshgen
    oracle.build()
    m = meshgen.kuhn_cube_mesh(args.N, seed=0)
    # calibrate: choose a per-step sample so the whole run takes about two minutes
    probe = min(50_000, m.nme)
    t0 = time.perf_counter()
    oracle.assemble(oracle.STIFF, m.q, np.ascontiguousarray(m.me[:, :probe]))
    rate = probe / (time.perf_counter() - t0)
    budget = 120.0 / max(1, args.steps + args.warmup)
    S = int(min(m.nme, max(10_000, rate * budget)))
    me = np.ascontiguousarray(m.me[:, :S])
    for k in range(args.warmup):
        t0 = time.perf_counter()
        oracle.assemble(oracle.STIFF, m.q, me)
        tw = time.perf_counter() - t0
        if k == 0 and tw > 1.3 * budget and args.warmup > 1:
            # the sort grows faster than linearly: shrink the sample to the step budget
            S = int(max(10_000, S * budget / tw))
            me = np.ascontiguousarray(m.me[:, :S])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.assemble(oracle.STIFF, m.q, me)
    dt = time.perf_counter() - t0
    value = S * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {**workload_config(args.N), "strategy": "oracle",
                                            "parallelism": "host, one thread"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"each step: the first {S:,} of the {m.nme:,} randomly ordered "
                                       "tets (element loop + triplet sort-and-sum, FP64)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ replicas (N > 1)
def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, steps: int, total_ms_max: float) -> float:
    """Whole-job throughput in millions of units per second: every rank processes its own
    copy of the workload, so the job processes world * units per step, in the time of the
    slowest rank."""
    return units_per_rank * world * steps / (total_ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------ GPU arm
def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1401_3301_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(form):
    """DRAM bytes per launch of the chunk kernel from the committed ncu summary, if the
    kernel sources are unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        ent = t[form]
        if ent.get("source_hash") != kernel_source_hash():
            return None
        return ent["bytes_per_launch"] * ent.get("scale_to_workload", 1.0)
    except Exception:
        return None


def chunk_algorithmic_bytes(p, prec, info, points=None):
    """Bytes the chunk kernel must move per launch: its plan records (read once), the
    FP64 coordinates (each point once: every vertex, or for P_k only the element
    vertices), the owned CSR values and the partial sums it writes; counts are exact,
    from the plan."""
    d = p.d
    npts = p.nq if points is None else points
    sT = 8 if prec == 0 else 4
    lv, le = info["local_vertices"], info["local_edges"]
    pv, pe = info["partial_vertices"], info["partial_edges"]
    reads = info["plan_bytes"] + 8 * d * npts
    writes = (lv - pv) * sT + (le - pe) * 2 * sT + (pv + pe) * 8
    return reads + writes


def fp64_instr_per_tet():
    """FP64-pipe instructions (DADD + DMUL + DFMA) per tet of the FP64 chunk kernel and
    their mix: ncu-counted when the committed profile matches the current kernel sources,
    else the count from the source (edges 9, cofactors 18, det 3, 1/(6|det|) 5, Gram 18,
    scaling 6, row sums 8, about 8 incidence sums) and no mix."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            ent = json.load(f)["f64"]
        if ent.get("source_hash") == kernel_source_hash() and "fp64_instr_per_tet" in ent:
            return (float(ent["fp64_instr_per_tet"]), "ncu (profiles/traffic.json)",
                    ent.get("fp64_instr_mix_per_tet"))
    except Exception:
        pass
    return 75.0, "from source", None


# FP64 issue rates measured on this GB300 with 8 independent dependency chains per
# thread (G instr/s at 2070 MHz): DFMA reaches 2 per SM per clock, DADD and DMUL only
# about 1.6, so a kernel's attainable FP64 rate depends on its instruction mix.
FP64_MEASURED_RATE = {"dfma": 599.0, "dadd": 505.0, "dmul": 505.0}


def fp64_mix_peak(mix):
    """Attainable FP64 instructions/s (G/s) for an instruction mix {op: per tet}."""
    total = sum(mix.values())
    return total / sum(n / FP64_MEASURED_RATE[k] for k, n in mix.items())


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1401_3301_gb300 import build_ext, fe, meshgen
    if rank == 0:
        build_ext.build()
    if world > 1:
        torch.distributed.barrier()
    fe.lib()
    m = meshgen.kuhn_cube_mesh(args.N, seed=0)
    q = torch.from_numpy(m.q).cuda()
    me = torch.from_numpy(m.me).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = fe.fe_pattern(q, me)
    pattern_ms = (time.perf_counter() - t0) * 1e3
    strategy = {"chunked": fe.REASM_CHUNKED, "gather": fe.REASM_GATHER, "atomic": fe.REASM_ATOMIC}[args.strategy]
    p.set_strategy(strategy)
    info = p.plan_info()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    hbm_peak, peak_src, sm_max = measured_peaks()
    stream = torch.cuda.current_stream()
    # per form: the autotuned pattern (chunk size, record layout, threads; untimed, cached)
    from paper_1401_3301_gb300 import tune
    pats, tuning = {}, {}
    pinned = json.loads(args.tuning) if args.tuning else {}
    for prec_name, prec in (("f64", fe.F64), ("f32", fe.F32), ("f64x", fe.F64X)):
        if args.strategy == "chunked" and prec_name in pinned:
            cfg = pinned[prec_name]
            pats[prec_name] = fe.fe_pattern(q, me, flags=fe.PATTERN_CHUNK(cfg["chunk"]) | cfg.get("layout", 0))
            pats[prec_name].set_threads(cfg.get("threads", 256))
            tuning[prec_name] = {"chunk": cfg["chunk"], "layout": cfg.get("layout", 0),
                                 "threads": cfg.get("threads", 256), "strategy": "chunked", "pinned": True}
        elif args.strategy == "chunked" and not args.no_tune:
            best = tune.autotune(q, me, "stiff", prec)
            pats[prec_name] = tune.tuned_pattern(q, me, "stiff", prec)
            tuning[prec_name] = {k: best[k] for k in ("chunk", "layout", "threads", "strategy")}
        else:
            pats[prec_name] = p
    sampler = ClockSampler(local)
    forms = {}
    sampler.start()
    for prec_name, prec in (("f64", fe.F64), ("f32", fe.F32), ("f64x", fe.F64X)):
        p = pats[prec_name]
        info = p.plan_info()
        T = torch.float32 if prec == fe.F32 else torch.float64
        vals = torch.empty(p.nnz, dtype=T, device="cuda")
        for _ in range(args.warmup):
            fe.fe_assemble_stiff(p, q, prec=prec, vals=vals)
        p.check()
        p.profile(True)
        p.profile_read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            fe.fe_assemble_stiff(p, q, prec=prec, vals=vals)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = max_over_ranks(float(sum(step_ms)), world, "cuda")
        prof = p.profile_read()
        p.profile(False)
        p.check()
        launches = int(sum(n for _, n in prof.values()))
        dom = max(prof, key=lambda k: prof[k][0])
        dom_ms = prof[dom][0] / prof[dom][1]
        abytes = chunk_algorithmic_bytes(p, fe.F64 if prec == fe.F64X else prec, info)
        achieved = abytes / (dom_ms * 1e-3) / 1e9
        traffic = committed_traffic(prec_name)
        roof_hbm = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic,
                    "algorithmic_bytes_per_launch": abytes, "kernel_ms": dom_ms,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                    else "fallback 6.8 TB/s"}
        value = replica_throughput(p.nme, world, args.steps, total_ms)
        forms[prec_name] = {"value": value, "ms_per_step": total_ms / args.steps,
                            "step_ms_median": statistics.median(step_ms), "kernels": {
                                k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in prof.items()},
                            "roofline_hbm": roof_hbm, "gpu_launches": launches}
        # path-level effective bandwidth with the per-tet bytes of the method (compulsory + slot map)
        per_tet = 94.3 if prec == fe.F32 else 104.4
        forms[prec_name]["path_effective"] = {
            "bytes_per_tet": per_tet, "GBps": per_tet * p.nme / (forms[prec_name]["ms_per_step"] * 1e-3) / 1e9}
        forms[prec_name]["path_effective"]["frac"] = forms[prec_name]["path_effective"]["GBps"] / hbm_peak
        if prec == fe.F64:
            clock = sm_max
            ipt, counted, mix = fp64_instr_per_tet()
            instr = ipt * p.nme
            peak_ops = FP64_PIPE_PER_SM_CLK * SM_COUNT * clock * 1e6 / 1e9
            achieved_ops = instr / (dom_ms * 1e-3) / 1e9
            forms[prec_name]["roofline_alu"] = {
                "bound": "alu", "kernel": dom, "achieved": achieved_ops,
                "peak": peak_ops, "unit": "G FP64 instr/s",
                "frac": achieved_ops / peak_ops, "traffic": traffic,
                "instr_per_tet": ipt, "counted": counted,
                "peak_source": f"{FP64_PIPE_PER_SM_CLK:.0f} FP64 instr/SM/clk x {SM_COUNT} SMs x {clock:.0f} MHz"}
            if mix:
                mp = fp64_mix_peak(mix)
                forms[prec_name]["roofline_alu"]["mix"] = {
                    "per_tet": mix, "attainable": mp, "frac": achieved_ops / mp,
                    "rates": FP64_MEASURED_RATE,
                    "source": "issue-rate microbenchmark (8 independent chains per thread)"}
    clocks = sampler.stop()

    # end-to-end through the public API with host buffers (selected form)
    prec = fe.F64 if args.prec == "f64" else fe.F32
    p = pats[args.prec]
    info = p.plan_info()
    T = torch.float64 if prec == fe.F64 else torch.float32
    # fe_assemble_stiff_host: every step uploads q and downloads the values through the
    # pattern's pipeline (step k's assembly beside step k+1's upload and k-1's download)
    q_host = torch.from_numpy(m.q).pin_memory()
    vals_host = [torch.empty(p.nnz, dtype=T).pin_memory() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 30))
    for k in range(4):
        fe.fe_assemble_stiff_host(p, q_host, vals_host[k % 2], prec=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(e2e_steps):
        fe.fe_assemble_stiff_host(p, q_host, vals_host[k % 2], prec=prec)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e = {"value": p.nme * world / (e2e_ms * 1e-3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(q_host.numel() * 8),
           "d2h_bytes_per_step": int(vals_host[0].numel() * vals_host[0].element_size()),
           "ms_per_step": e2e_ms, "steps": e2e_steps, "call": "fe_assemble_stiff_host (pinned host q in, "
                                                              "host values out, successive steps overlapped)"}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    sel = forms[args.prec]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(m, args.cpu_sample)
    roof = sel["roofline_alu"] if args.prec == "f64" else sel["roofline_hbm"]
    line = {"metric": METRIC, "value": sel["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sel["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {**workload_config(args.N), "strategy": args.strategy, "form": args.prec,
                       "tuning": tuning or "default pattern",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "nnz": p.nnz, "pattern_build_ms": pattern_ms, "plan": info},
            "roofline": roof, "forms": forms, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": sel["gpu_launches"], "clocks": clocks}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ other configurations
def _timed(fn, steps, warmup, flush=None):
    """Median and mean ms of fn over `steps` calls (CUDA events; optional L2 flush, untimed)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        if flush is not None:
            flush.fill_(1)
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    t = [a.elapsed_time(b) for a, b in ev]
    return statistics.median(t), sum(t) / len(t)


def run_other(args):
    import torch
    from paper_1401_3301_gb300 import build_ext, fe, meshgen
    build_ext.build()
    fe.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, W = args.steps, args.warmup
    out = {"workload": args.workload, "data": "synthetic", "steps": K, "warmup": W, "n_gpus": 1,
           "higher_is_better": True, "forms": {}}
    if args.workload in ("mass", "wmass"):
        m = meshgen.kuhn_cube_mesh(args.N, seed=0)
        q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        p = fe.fe_pattern(q, me)
        wv = torch.from_numpy(meshgen.vertex_weights(0, m.nq)).cuda()
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            w = wv.to(T)
            fn = (lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals)) if args.workload == "mass" else \
                 (lambda: fe.fe_assemble_wmass(p, q, w, fe.COEF_P1, prec=prec, vals=vals))
            med, mean = _timed(fn, K, W, flush)
            p.check()
            out["forms"][name] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
        out.update(metric=f"3D P1 {'mass' if args.workload == 'mass' else 'weighted mass (P1 vertex weight)'} "
                          "Mtets/s, fixed pattern", unit="Mtets/s",
                   config=workload_config(args.N, "mass" if args.workload == "mass"
                                          else "weighted mass (P1 vertex weight)"))
    elif args.workload == "general":
        # convection-diffusion-reaction operator (non-symmetric), per-element and per-vertex
        # coefficient sets of 16 values each
        m = meshgen.kuhn_cube_mesh(args.N, seed=0)
        q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        p = fe.fe_pattern(q, me)
        c0 = meshgen.general_coefficients(0, 3, m.nme)
        c1 = meshgen.general_coefficients(1, 3, m.nq)
        order = p.element_order().long().cpu().numpy()
        c0i = np.ascontiguousarray(c0[order])
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            res = {}
            for label, arr, kind in (("p0_internal", c0i, fe.COEF_P0_INTERNAL), ("p0", c0, fe.COEF_P0),
                                     ("p1", c1, fe.COEF_P1)):
                cf = torch.from_numpy(arr).cuda().to(T)
                med, mean = _timed(lambda: fe.fe_assemble_general(p, q, cf, kind, prec=prec, vals=vals), K, W,
                                   flush)
                p.check()
                res[label] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
            out["forms"][name] = {"value": res["p0_internal"]["value"], "coefficients": res}
        out.update(metric="3D P1 general operator -div(A grad u) + div(b u) + c.grad u + a0 u (non-symmetric) "
                          "Mtets/s, fixed pattern", unit="Mtets/s",
                   config=workload_config(args.N, "general operator (Eq. EDP)"))
    elif args.workload == "pk":
        # 3D P_k mass (App. D) at the largest size of the paper's P_k table, about 10^6 nodes:
        # k N = 100 cells per side on the fine lattice, (kN+1)^3 nodes, for k = 1..6
        hbm_peak, _, _ = measured_peaks()
        for k in range(1, 7):
            N = {1: 100, 2: 50, 3: 33, 4: 25, 5: 20, 6: 17}[k]
            m = meshgen.pk_mesh(3, N, k, seed=0)
            q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p = fe.fe_pk_pattern(q, me, k)
            pms = (time.perf_counter() - t0) * 1e3
            info = p.plan_info()
            res = {"N": N, "nodes": m.nq, "tets": m.nme, "nnz": p.nnz, "chunk": info["chunk"],
                   "pattern_build_ms": pms}
            for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                                  ("f64x", fe.F64X, torch.float64)):
                vals = torch.empty(p.nnz, dtype=T, device="cuda")
                med, mean = _timed(lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals), K, W, flush)
                p.check()
                sT = 4 if prec == fe.F32 else 8
                abytes = chunk_algorithmic_bytes(p, fe.F64 if prec == fe.F64X else prec, info, points=(N + 1) ** 3)
                res[name] = {"ms_per_step": mean, "ms_median": med, "Mnodes_per_s": m.nq / (mean * 1e-3) / 1e6,
                             "Mnnz_per_s": p.nnz / (mean * 1e-3) / 1e6,
                             "algorithmic_bytes": abytes, "GBps": abytes / (mean * 1e-3) / 1e9,
                             "hbm_frac": abytes / (mean * 1e-3) / 1e9 / hbm_peak, "value_bytes": p.nnz * sT}
            out["forms"][f"k{k}"] = res
            del p, vals, q, me
        out["forms"]["f64"] = {"value": out["forms"]["k2"]["f64"]["Mnodes_per_s"]}
        out.update(metric="3D P_k mass (App. D), k = 1..6 at about 10^6 nodes: M nodes/s, fixed pattern "
                          "(value: k = 2, FP64)", unit="M nodes/s",
                   config={"workload": "Kuhn cube, P_k lattice nodes, kN ~ 100 (about 1.03e6 nodes), jitter 0.15h, "
                                       "elements permuted", "hbm_peak_GBps": hbm_peak})
    elif args.workload == "boundary":
        # facet (boundary) mass and P1-weighted mass on a large triangulated surface in 3D,
        # as generated (random vertex numbering) and after fe_morton_vertex_order
        N = 2000 if args.N == 100 else args.N
        m = meshgen.surface_mesh(N, seed=0)
        q0, f0 = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        wv0 = torch.from_numpy(meshgen.vertex_weights(0, m.nq)).cuda()
        order = fe.fe_morton_vertex_order(q0)
        q1, f1 = fe.fe_apply_vertex_order(q0, f0, order)
        numberings = {"as_generated": (q0, f0, wv0), "morton": (q1, f1, wv0[order.long()])}
        pms = {}
        for label_n, (q, f, wv) in numberings.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p = fe.fe_boundary_pattern(q, f)
            pms[label_n] = (time.perf_counter() - t0) * 1e3
            for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                                  ("f64x", fe.F64X, torch.float64)):
                vals = torch.empty(p.nnz, dtype=T, device="cuda")
                w = wv.to(T)
                res = {}
                for label, fn in (("mass", lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals)),
                                  ("wmass_p1", lambda: fe.fe_assemble_wmass(p, q, w, fe.COEF_P1, prec=prec,
                                                                            vals=vals))):
                    med, mean = _timed(fn, K, W, flush)
                    p.check()
                    res[label] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
                out["forms"].setdefault(name, {"value": None, "numbering": {}})["numbering"][label_n] = res
            nnz = p.nnz
            del p
        for name in ("f64", "f32", "f64x"):
            out["forms"][name]["value"] = out["forms"][name]["numbering"]["morton"]["mass"]["value"]
        out.update(metric="3D surface (facet) mass and P1-weighted mass, Mtris/s, fixed pattern (value: Morton "
                          "vertex numbering, mass)", unit="Mtris/s",
                   config={"workload": f"height-field surface over the unit square, N={N} ({m.nme:,} triangles, "
                                       f"{m.nq:,} vertices), jitter 0.2h, vertices and elements permuted",
                           "nnz": nnz, "pattern_build_ms": pms})
    elif args.workload == "elas":
        N = 80 if args.N == 100 else args.N
        m = meshgen.kuhn_cube_mesh(N, seed=0)
        q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        t0 = time.perf_counter()
        p = fe.fe_pattern(q, me, m=3)
        pms = (time.perf_counter() - t0) * 1e3
        lam0, mu0 = meshgen.lame_from_young(1.0, 0.3)
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            lam = torch.tensor([lam0], dtype=T, device="cuda")
            mu = torch.tensor([mu0], dtype=T, device="cuda")
            med, mean = _timed(lambda: fe.fe_assemble_elas(p, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR,
                                                          prec=prec, vals=vals), K, W, flush)
            p.check()
            # rigid-mode residual: K r for the 6 rigid modes, relative to |K| |r|
            rp, ci = p.csr()
            rows = torch.repeat_interleave(torch.arange(p.n, device="cuda"), (rp[1:] - rp[:-1]).long())
            X = q.T.double()
            res = 0.0
            for mode in range(6):
                r = torch.zeros((m.nq, 3), dtype=torch.float64, device="cuda")
                if mode < 3:
                    r[:, mode] = 1.0
                else:
                    axis = torch.zeros(3, dtype=torch.float64, device="cuda")
                    axis[mode - 3] = 1.0
                    r = torch.linalg.cross(axis.expand_as(X), X)
                r = r.reshape(-1)
                y = torch.zeros(p.n, dtype=torch.float64, device="cuda")
                y.index_add_(0, rows, vals.double() * r[ci.long()])
                res = max(res, float(y.abs().max() / (vals.double().abs().max() * r.abs().max())))
            out["forms"][name] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6,
                                  "rigid_mode_residual": res}
        out.update(metric="3D P1 linear elasticity (12x12 element blocks) Mtets/s, fixed pattern", unit="Mtets/s",
                   config={**workload_config(N, "linear elasticity"), "E": 1.0, "nu": 0.3, "nnz": p.nnz,
                           "pattern_build_ms": pms})
    elif args.workload == "2d":
        m = meshgen.square_mesh(100, seed=0)
        q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        p = fe.fe_pattern(q, me)
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            v1 = torch.empty(p.nnz, dtype=T, device="cuda")
            v2 = torch.empty(p.nnz, dtype=T, device="cuda")

            def step():
                fe.fe_assemble_mass(p, q, prec=prec, vals=v1)
                fe.fe_assemble_stiff(p, q, prec=prec, vals=v2)
            step()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            med, mean = _timed(g.replay, K, W)
            out["forms"][name] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
        out.update(metric="2D P1 mass + stiffness Mtris/s (both matrices per step, CUDA graph)", unit="Mtris/s",
                   config={"workload": "unit square N=100, 20,000 triangles, 10,201 vertices, jitter 0.2h, "
                                       "vertices and elements permuted", "nnz": p.nnz})
    elif args.workload == "batched":
        sizes = meshgen.batch_sizes(0, 256, 16, 512)
        meshes = [meshgen.square_mesh(int(n), seed=b + 1) for b, n in enumerate(sizes)]
        qs = [torch.from_numpy(mm.q).cuda() for mm in meshes]
        mes = [torch.from_numpy(mm.me).cuda() for mm in meshes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = fe.fe_batch_pattern(qs, mes)
        pms = (time.perf_counter() - t0) * 1e3
        vo, eo, _ = fe.fe_batch_offsets(p)
        qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
        fe.fe_batch_gather_q(p, qs, mes, qu)
        del qs, mes
        ntri = int(eo[-1])
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            w = torch.ones(ntri, dtype=T, device="cuda")
            s = torch.empty(p.nnz, dtype=T, device="cuda")
            mm_ = torch.empty(p.nnz, dtype=T, device="cuda")
            torch.cuda.manual_seed(0)

            def step():
                # fresh lognormal(0, 1) weights, drawn in FP32 (input data: an FP64 normal
                # generator would cost more FP64 work than the assembly) and widened to the form
                w.copy_(torch.randn(w.shape, device="cuda", dtype=torch.float32).exp_())
                fe.fe_assemble_stiff(p, qu, w, fe.COEF_P0_INTERNAL, prec=prec, vals=s)
                fe.fe_assemble_wmass(p, qu, w, fe.COEF_P0_INTERNAL, prec=prec, vals=mm_)
            step()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            med, mean = _timed(g.replay, K, W)
            p.check()
            out["forms"][name] = {"ms_per_step": mean, "ms_median": med, "value": ntri / (mean * 1e-3) / 1e6}
        out.update(metric="Batched 2D weighted mass + stiffness reassembly with fresh lognormal weights, "
                          "Mtris/s (CUDA graph replay)", unit="Mtris/s",
                   config={"workload": f"256 jittered unit-square meshes, N uniform in [16, 512] "
                                       f"({ntri:,} triangles, {int(vo[-1]):,} vertices)", "nnz": p.nnz,
                           "pattern_build_ms": pms})
    elif args.workload == "diff":
        N = 64 if args.N == 100 else args.N
        m = meshgen.kuhn_cube_mesh(N, seed=0)
        q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
        p = fe.fe_pattern(q, me)
        w64 = torch.from_numpy(meshgen.element_weights(0, m.nme)).cuda()
        u64, v64 = (torch.from_numpy(x).cuda() for x in meshgen.random_vectors(0, m.nq))
        for name, prec, T in (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32),
                              ("f64x", fe.F64X, torch.float64)):
            w, u, v = w64.to(T), u64.to(T), v64.to(T)
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            L = torch.empty(1, dtype=T, device="cuda")
            dw = torch.empty(m.nme, dtype=T, device="cuda")
            dq = torch.empty((3, m.nq), dtype=T, device="cuda")

            def step():
                fe.fe_assemble_stiff(p, q, w, fe.COEF_P0, prec=prec, vals=vals)
                fe.fe_assemble_stiff_backward(p, q, w, fe.COEF_P0, u, v, L, dw, dq, prec=prec)
            med, mean = _timed(step, K, W, flush)
            p.check()
            out["forms"][name] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
        out.update(metric="3D stiffness K(w) forward + backward (L = u^T K v, dL/dw, dL/dq) Mtets/s",
                   unit="Mtets/s", config={**workload_config(N, "stiffness forward + backward")})
    out["value"] = out["forms"]["f64"]["value"]
    out["dtype"] = "f64"
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "stiffness":
        run_other(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

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
    ap.add_argument("--no-secondary", action="store_true",
                    help="headline only: skip the other configurations' block")
    ap.add_argument("--batch-meshes", type=int, default=256,
                    help="--workload batched: meshes in the batch (default 256; fewer for a profiler capture)")
    ap.add_argument("--replays", type=int, default=1000,
                    help="--workload batched: timed graph replays (default 1000)")
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


def cpu_baseline(m, sample, reps=5):
    """The FP64 oracle on the host cores, on the headline mesh:
    - value: fixed-pattern reassembly (every element's local matrix, then each nonzero's
      sum over the oracle's own slot map), like for like with the GPU headline, on all
      cores, the whole mesh, median of `reps` runs;
    - beside it: the same on one thread (one run), and the full assembly (element loop,
      triplet sort, sums: the `sparse` construction) on all cores over the whole mesh
      and on one thread over the first `sample` tets (one run each).
    The slot map is built once, untimed (like the GPU pattern)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    ptr, n2s = oracle.slot_map(m.me, m.nq)
    setup = time.perf_counter() - t0

    def timed(fn):
        t = time.perf_counter()
        fn()
        return time.perf_counter() - t
    reasm = lambda: oracle.reassemble(oracle.STIFF, m.q, m.me, ptr, n2s)
    timed(reasm)  # warm-up (page faults of the value arrays)
    runs = sorted(timed(reasm) for _ in range(reps))
    med = statistics.median(runs)
    full_all = timed(lambda: oracle.assemble(oracle.STIFF, m.q, m.me))
    oracle.set_threads(1)
    reasm_1 = timed(reasm)
    S = min(sample, m.nme)
    me_s = np.ascontiguousarray(m.me[:, :S])
    full_1 = timed(lambda: oracle.assemble(oracle.STIFF, m.q, me_s))
    del ptr, n2s
    rate = lambda n, t: n / t / 1e6
    return {"value": rate(m.nme, med), "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
            "sample": f"the whole {m.nme:,}-tet mesh: fixed-pattern reassembly (element loop + sums over the "
                      f"oracle's slot map, FP64), {cores} threads, median of {reps} runs "
                      f"({', '.join(f'{x:.3f}' for x in runs)} s; slot map built once in {setup:.1f} s, untimed)",
            "fixed_pattern_1_thread": {"value": rate(m.nme, reasm_1), "cores": 1, "seconds": reasm_1,
                                       "sample": "whole mesh, one run"},
            "full_assembly": {"value": rate(m.nme, full_all), "cores": cores, "seconds": full_all,
                              "sample": "whole mesh (element loop + triplet sort-and-sum into CSR), one run"},
            "full_assembly_1_thread": {"value": rate(S, full_1), "cores": 1, "seconds": full_1,
                                       "sample": f"first {S:,} of the {m.nme:,} randomly ordered tets, one run"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1401_3301_gb300 import meshgen
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
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
                                            "parallelism": f"host, {cores} threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
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


def committed_profile(form, cfg):
    """The committed ncu counters (profiles/traffic.json) of the form's chunk kernel in the
    configuration (chunk, record layout, threads) of this run's pattern, if the kernel
    sources are unchanged since they were taken; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            entries = json.load(f)[form]
    except (OSError, ValueError, KeyError):
        return None
    for ent in entries:
        got = ent.get("configuration", {})
        if ent.get("source_hash") == kernel_source_hash() and all(
                got.get(k) == cfg.get(k) for k in ("chunk", "layout", "threads")):
            return ent
    return None


def committed_traffic(form, cfg):
    """DRAM bytes (read + write) per launch of the chunk kernel at this workload's size,
    from the committed counters (scaled from the captured mesh by the number of tets)."""
    ent = committed_profile(form, cfg)
    return None if ent is None else ent["bytes_per_launch"] * ent.get("scale_to_workload", 1.0)


def chunk_algorithmic_bytes(p, prec, info, points=None, block=1, matrices=1, extra_reads=0):
    """Bytes the chunk kernel must move per launch: its plan records (read once), the
    FP64 coordinates (each point once: every vertex, or for P_k only the element
    vertices), the owned CSR values and the partial sums it writes (block values per
    vertex or edge entry: m * m for vector problems; `matrices` matrices at once), plus
    extra_reads (coefficients); counts are exact, from the plan."""
    d = p.d
    npts = p.nq if points is None else points
    sT = 4 if prec == 1 else 8  # CSR values: FP32 form float, FP64 and F64X double
    sP = 4 if prec == 1 else 8  # partials: FP32 float, FP64 double, F64X float pair
    lv, le = info["local_vertices"], info["local_edges"]
    pv, pe = info["partial_vertices"], info["partial_edges"]
    reads = info["plan_bytes"] + 8 * d * npts + extra_reads
    writes = ((lv - pv) * sT + (le - pe) * 2 * sT + (pv + pe) * sP) * block * matrices
    return reads + writes


def fixup_algorithmic_bytes(prec, info):
    """Bytes the fixup must move per launch: per shared vertex / edge its list bound (4 B)
    and destinations (8 B), its partial sums (4 B each in the FP32 form, else 8 B), and the
    values it writes (one per shared vertex, two per shared edge)."""
    nsh_v, nsh_e = info["shared_vertices"], info["shared_edges"]
    npart = info["partial_vertices"] + info["partial_edges"]
    sT = 4 if prec == 1 else 8
    sP = 4 if prec == 1 else 8
    return 4 * (nsh_v + nsh_e + 1) + 8 * (nsh_v + nsh_e) + sP * npart + sT * (nsh_v + 2 * nsh_e)


def fp64_instr_per_tet(cfg):
    """FP64-pipe instructions (DADD + DMUL + DFMA) per tet of the FP64 chunk kernel and
    their mix: ncu-counted when a committed profile matches the current kernel sources and
    configuration, else the count from the source (edges 9, cofactors 18, det 3,
    1/(6|det|) 5, Gram 18, scaling 6, row sums 8, about 8 incidence sums) and no mix."""
    ent = committed_profile("f64", cfg)
    if ent is not None and "fp64_instr_per_tet" in ent:
        return (float(ent["fp64_instr_per_tet"]), "ncu (profiles/traffic.json)", ent.get("fp64_instr_mix_per_tet"))
    return 75.0, "from source", None


# FP64 issue rate measured on this GB300 by a microbenchmark (1216 blocks of 256
# threads, 8 independent dependency chains per thread, SM clock 1995-2070 MHz): DADD,
# DMUL and DFMA alike issue at 529 G instr/s, 0.84 of the 2 per SM per clock at 2070 MHz.
FP64_MEASURED_RATE = 529.0


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
        traffic = committed_traffic(prec_name, tuning.get(prec_name, {}))
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
        if "fixup" in prof:
            fx_ms = prof["fixup"][0] / prof["fixup"][1]
            fx_bytes = fixup_algorithmic_bytes(prec, info)
            forms[prec_name]["roofline_fixup"] = {
                "bound": "hbm", "kernel": "fixup", "achieved": fx_bytes / (fx_ms * 1e-3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "frac": fx_bytes / (fx_ms * 1e-3) / 1e9 / hbm_peak,
                "algorithmic_bytes_per_launch": fx_bytes, "kernel_ms": fx_ms,
                "share_of_step": fx_ms / (total_ms / args.steps)}
        # path-level effective bandwidth with the per-tet bytes of the method (compulsory + slot map)
        per_tet = 94.3 if prec == fe.F32 else 104.4
        forms[prec_name]["path_effective"] = {
            "bytes_per_tet": per_tet, "GBps": per_tet * p.nme / (forms[prec_name]["ms_per_step"] * 1e-3) / 1e9}
        forms[prec_name]["path_effective"]["frac"] = forms[prec_name]["path_effective"]["GBps"] / hbm_peak
        if prec == fe.F64:
            clock = sm_max
            ipt, counted, mix = fp64_instr_per_tet(tuning.get(prec_name, {}))
            instr = ipt * p.nme
            peak_ops = FP64_PIPE_PER_SM_CLK * SM_COUNT * clock * 1e6 / 1e9
            achieved_ops = instr / (dom_ms * 1e-3) / 1e9
            forms[prec_name]["roofline_alu"] = {
                "bound": "alu", "kernel": dom, "achieved": achieved_ops,
                "peak": peak_ops, "unit": "G FP64 instr/s",
                "frac": achieved_ops / peak_ops, "traffic": traffic,
                "instr_per_tet": ipt, "counted": counted,
                "peak_source": f"{FP64_PIPE_PER_SM_CLK:.0f} FP64 instr/SM/clk x {SM_COUNT} SMs x {clock:.0f} MHz"}
            forms[prec_name]["roofline_alu"]["measured"] = {
                "attainable": FP64_MEASURED_RATE, "frac": achieved_ops / FP64_MEASURED_RATE,
                "per_tet": mix,
                "source": "FP64 issue-rate microbenchmark: DADD, DMUL and DFMA alike (8 independent "
                          "chains per thread, SM clock 1995-2070 MHz)"}
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
    workloads = None
    if world == 1 and not args.no_secondary:
        del pats
        torch.cuda.empty_cache()
        workloads = secondary_workloads(fe, torch, flush, hbm_peak)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(m, args.cpu_sample)
    roof = sel["roofline_hbm"]
    line = {"metric": METRIC, "value": sel["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sel["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {**workload_config(args.N), "strategy": args.strategy, "form": args.prec,
                       "tuning": tuning or "default pattern",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "nnz": p.nnz, "pattern_build_ms": pattern_ms, "plan": info},
            "roofline": roof, "roofline_alu": sel.get("roofline_alu"), "forms": forms, "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": sel["gpu_launches"], "clocks": clocks, "workloads": workloads}
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


def _forms(fe, torch):
    return (("f64", fe.F64, torch.float64), ("f32", fe.F32, torch.float32), ("f64x", fe.F64X, torch.float64))


def _kernels(p, fn, steps=5, flush=None):
    """{kernel: ms per launch} of the library's kernels over `steps` calls of fn on
    pattern p (fe_profile: CUDA events around each launch; L2 flushed between calls)."""
    p.profile(True)
    p.profile_read()
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1)
        fn()
    prof = p.profile_read()
    p.profile(False)
    return {k: v[0] / v[1] for k, v in prof.items() if v[1]}


def _entry(units, ms_mean, ms_median, kern=None, abytes=None, hbm_peak=None, dominant="chunk", **extra):
    """One form's result: throughput, step time, per-kernel times and, for a chunk kernel
    with a known byte count, its HBM roofline fraction (algorithmic bytes / kernel time)."""
    e = {"value": units / (ms_mean * 1e-3) / 1e6, "ms_per_step": ms_mean, "ms_median": ms_median}
    if kern:
        e["kernels_ms"] = kern
        if abytes is not None and dominant in kern:
            gbs = abytes / (kern[dominant] * 1e-3) / 1e9
            e["roofline"] = {"bound": "hbm", "kernel": dominant, "algorithmic_bytes_per_launch": abytes,
                             "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak}
    e.update(extra)
    return e


def wl_mass(fe, torch, K, W, flush, hbm_peak, N=100, which=("mass", "wmass")):
    """3D P1 mass and P1-weighted mass, fixed pattern (the headline mesh)."""
    from paper_1401_3301_gb300 import meshgen
    m = meshgen.kuhn_cube_mesh(N, seed=0)
    q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
    p = fe.fe_pattern(q, me)
    info = p.plan_info()
    wv = torch.from_numpy(meshgen.vertex_weights(0, m.nq)).cuda()
    out = {}
    for op in which:
        res = {}
        for name, prec, T in _forms(fe, torch):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            w = wv.to(T)
            fn = (lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals)) if op == "mass" else \
                 (lambda: fe.fe_assemble_wmass(p, q, w, fe.COEF_P1, prec=prec, vals=vals))
            med, mean = _timed(fn, K, W, flush)
            kern = _kernels(p, fn, flush=flush)
            p.check()
            ab = chunk_algorithmic_bytes(p, 0 if prec == fe.F64X else prec, info,
                                         extra_reads=0 if op == "mass" else 8 * m.nq)
            res[name] = _entry(m.nme, mean, med, kern, ab, hbm_peak)
        out[op] = {"metric": f"3D P1 {'mass' if op == 'mass' else 'weighted mass (P1 vertex weight)'} Mtets/s, "
                             "fixed pattern", "unit": "Mtets/s",
                   "config": workload_config(N, "mass" if op == "mass" else "weighted mass (P1 vertex weight)"),
                   "forms": res}
    return out


def wl_elas(fe, torch, K, W, flush, hbm_peak, N=80):
    """3D P1 linear elasticity, 3 dofs per vertex, E = 1, nu = 0.3, with the rigid-mode check."""
    from paper_1401_3301_gb300 import meshgen
    m = meshgen.kuhn_cube_mesh(N, seed=0)
    q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
    t0 = time.perf_counter()
    p = fe.fe_pattern(q, me, m=3)
    pms = (time.perf_counter() - t0) * 1e3
    info = p.plan_info()
    lam0, mu0 = meshgen.lame_from_young(1.0, 0.3)
    rp, ci = p.csr()
    rows = torch.repeat_interleave(torch.arange(p.n, device="cuda"), (rp[1:] - rp[:-1]).long())
    X = q.T.double()
    res = {}
    for name, prec, T in _forms(fe, torch):
        vals = torch.empty(p.nnz, dtype=T, device="cuda")
        lam = torch.tensor([lam0], dtype=T, device="cuda")
        mu = torch.tensor([mu0], dtype=T, device="cuda")
        fn = lambda: fe.fe_assemble_elas(p, q, lam, fe.COEF_SCALAR, mu, fe.COEF_SCALAR, prec=prec, vals=vals)
        med, mean = _timed(fn, K, W, flush)
        kern = _kernels(p, fn, flush=flush)
        p.check()
        # rigid-mode residual: K r for the 6 rigid modes, relative to |K| |r|
        resid = 0.0
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
            resid = max(resid, float(y.abs().max() / (vals.double().abs().max() * r.abs().max())))
        ab = chunk_algorithmic_bytes(p, 0 if prec == fe.F64X else prec, info, block=9)
        res[name] = _entry(m.nme, mean, med, kern, ab, hbm_peak, dominant="elas_chunk", rigid_mode_residual=resid)
    return {"metric": "3D P1 linear elasticity (12x12 element blocks) Mtets/s, fixed pattern", "unit": "Mtets/s",
            "config": {**workload_config(N, "linear elasticity"), "E": 1.0, "nu": 0.3, "nnz": p.nnz,
                       "pattern_build_ms": pms}, "forms": res}


def wl_2d(fe, torch, K, W, flush, hbm_peak, N=100):
    """2D P1 mass + stiffness (both matrices per step) in one CUDA graph."""
    from paper_1401_3301_gb300 import meshgen
    m = meshgen.square_mesh(N, seed=0)
    q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
    p = fe.fe_pattern(q, me)
    res = {}
    for name, prec, T in _forms(fe, torch):
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
        kern = _kernels(p, step)
        p.check()
        res[name] = _entry(m.nme, mean, med, kern)
    return {"metric": "2D P1 mass + stiffness Mtris/s (both matrices per step, CUDA graph)", "unit": "Mtris/s",
            "config": {"workload": f"unit square N={N}, {m.nme:,} triangles, {m.nq:,} vertices, jitter 0.2h, "
                                   "vertices and elements permuted", "nnz": p.nnz}, "forms": res}


def wl_batched(fe, torch, K, W, flush, hbm_peak, replays=1000, count=256):
    """The 256-mesh 2D batch: weighted mass + stiffness with fresh lognormal(0, 1)
    per-element weights every step, one fused persistent kernel (+ one fixup) on the
    pattern the autotuner picks for the batch, captured with the weight draw in a CUDA
    graph and replayed `replays` times (the time per replay is reported). The F64X form's
    fused kernel takes one block per chunk and runs one fixup per matrix."""
    from paper_1401_3301_gb300 import meshgen, tune
    sizes = meshgen.batch_sizes(0, count, 16, 512)
    meshes = [meshgen.square_mesh(int(n), seed=b + 1) for b, n in enumerate(sizes)]
    qs = [torch.from_numpy(mm.q).cuda() for mm in meshes]
    mes = [torch.from_numpy(mm.me).cuda() for mm in meshes]
    del meshes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p0 = fe.fe_batch_pattern(qs, mes)
    pms = (time.perf_counter() - t0) * 1e3
    vo, eo, _ = fe.fe_batch_offsets(p0)
    qu = torch.empty((2, int(vo[-1])), dtype=torch.float64, device="cuda")
    fe.fe_batch_gather_q(p0, qs, mes, qu)
    ntri = int(eo[-1])
    res, tuning = {}, {}
    for name, prec, T in _forms(fe, torch):
        w = torch.ones(ntri, dtype=T, device="cuda")

        def make(flags, _qs=qs, _mes=mes):
            return fe.fe_batch_pattern(_qs, _mes, flags=flags)
        best = tune.autotune(qu, torch.empty((3, ntri), device="meta"), "wmass_stiff", prec, w=w,
                             w_kind=fe.COEF_P0_INTERNAL, pattern=make, tag=f"batch{count}", reps=5)
        p = tune.tuned_pattern(qu, torch.empty((3, ntri), device="meta"), "wmass_stiff", prec, w=w,
                               w_kind=fe.COEF_P0_INTERNAL, pattern=make, tag=f"batch{count}", reps=5)
        tuning[name] = {k: best.get(k) for k in ("chunk", "layout", "threads", "persistent")}
        s_ = torch.empty(p.nnz, dtype=T, device="cuda")
        m_ = torch.empty(p.nnz, dtype=T, device="cuda")

        def assemble():
            fe.fe_assemble_wmass_stiff(p, qu, w, fe.COEF_P0_INTERNAL, prec=prec, vals_mass=m_, vals_stiff=s_)
        torch.cuda.manual_seed(0)

        def step():
            # fresh lognormal(0, 1) weights, drawn in FP32 (input data: an FP64 normal
            # generator would cost more FP64 work than the assembly) and widened to the form
            w.copy_(torch.randn(w.shape, device="cuda", dtype=torch.float32).exp_())
            assemble()
        step()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(W):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(replays):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        mean = e0.elapsed_time(e1) / replays
        kern = _kernels(p, assemble)
        p.check()
        info = p.plan_info()
        sT = 4 if prec == fe.F32 else 8
        ab = chunk_algorithmic_bytes(p, 0 if prec == fe.F64X else prec, info, matrices=2, extra_reads=sT * ntri)
        res[name] = _entry(ntri, mean, mean, kern, ab, hbm_peak, replays=replays,
                           launches_per_step=2 if prec != fe.F64X else 3)
    return {"metric": "Batched 2D weighted mass + stiffness reassembly with fresh lognormal weights, Mtris/s "
                      f"(CUDA graph, {replays} replays)", "unit": "Mtris/s",
            "config": {"workload": f"{count} jittered unit-square meshes, N uniform in [16, 512] ({ntri:,} "
                                   f"triangles, {int(vo[-1]):,} vertices)", "nnz": p0.nnz,
                       "pattern_build_ms": pms, "tuning": tuning, "replays": replays}, "forms": res}


def wl_diff(fe, torch, K, W, flush, hbm_peak, N=64):
    """3D stiffness K(w) forward + backward: L = u^T K(w) v, dL/dw, dL/dq."""
    from paper_1401_3301_gb300 import meshgen
    m = meshgen.kuhn_cube_mesh(N, seed=0)
    q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
    p = fe.fe_pattern(q, me)
    w64 = torch.from_numpy(meshgen.element_weights(0, m.nme)).cuda()
    u64, v64 = (torch.from_numpy(x).cuda() for x in meshgen.random_vectors(0, m.nq))
    res = {}
    for name, prec, T in _forms(fe, torch):
        w, u, v = w64.to(T), u64.to(T), v64.to(T)
        vals = torch.empty(p.nnz, dtype=T, device="cuda")
        L = torch.empty(1, dtype=T, device="cuda")
        dw = torch.empty(m.nme, dtype=T, device="cuda")
        dq = torch.empty((3, m.nq), dtype=T, device="cuda")

        def step():
            fe.fe_assemble_stiff(p, q, w, fe.COEF_P0, prec=prec, vals=vals)
            fe.fe_assemble_stiff_backward(p, q, w, fe.COEF_P0, u, v, L, dw, dq, prec=prec)
        med, mean = _timed(step, K, W, flush)
        kern = _kernels(p, step, flush=flush)
        p.check()
        res[name] = _entry(m.nme, mean, med, kern)
    return {"metric": "3D stiffness K(w) forward + backward (L = u^T K v, dL/dw, dL/dq) Mtets/s", "unit": "Mtets/s",
            "config": workload_config(N, "stiffness forward + backward"), "forms": res}


def wl_general(fe, torch, K, W, flush, hbm_peak, N=100):
    """3D P1 general operator (Eq. EDP), P0 records in internal and input order, P1 records."""
    from paper_1401_3301_gb300 import meshgen
    forms = {}
    # convection-diffusion-reaction operator (non-symmetric), per-element and per-vertex
    # coefficient sets of 16 values each
    m = meshgen.kuhn_cube_mesh(N, seed=0)
    q, me = torch.from_numpy(m.q).cuda(), torch.from_numpy(m.me).cuda()
    p = fe.fe_pattern(q, me)
    c0 = meshgen.general_coefficients(0, 3, m.nme)
    c1 = meshgen.general_coefficients(1, 3, m.nq)
    order = p.element_order().long().cpu().numpy()
    c0i = np.ascontiguousarray(c0[order])
    for name, prec, T in _forms(fe, torch):
        vals = torch.empty(p.nnz, dtype=T, device="cuda")
        res = {}
        for label, arr, kind in (("p0_internal", c0i, fe.COEF_P0_INTERNAL), ("p0", c0, fe.COEF_P0),
                                 ("p1", c1, fe.COEF_P1)):
            cf = torch.from_numpy(arr).cuda().to(T)
            med, mean = _timed(lambda: fe.fe_assemble_general(p, q, cf, kind, prec=prec, vals=vals), K, W,
                               flush)
            p.check()
            res[label] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
        forms[name] = {"value": res["p0_internal"]["value"], "coefficients": res}
    return dict(forms=forms, metric="3D P1 general operator -div(A grad u) + div(b u) + c.grad u + a0 u "
                                    "(non-symmetric) Mtets/s, fixed pattern", unit="Mtets/s",
                config=workload_config(N, "general operator (Eq. EDP)"))


def wl_pk(fe, torch, K, W, flush, hbm_peak):
    """3D P_k mass (App. D), k = 1..6 at about 10^6 nodes."""
    from paper_1401_3301_gb300 import meshgen
    forms = {}
    # 3D P_k mass (App. D) at the largest size of the paper's P_k table, about 10^6 nodes:
    # k N = 100 cells per side on the fine lattice, (kN+1)^3 nodes, for k = 1..6
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
        for name, prec, T in _forms(fe, torch):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            med, mean = _timed(lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals), K, W, flush)
            p.check()
            sT = 4 if prec == fe.F32 else 8
            abytes = chunk_algorithmic_bytes(p, fe.F64 if prec == fe.F64X else prec, info, points=(N + 1) ** 3)
            res[name] = {"ms_per_step": mean, "ms_median": med, "Mnodes_per_s": m.nq / (mean * 1e-3) / 1e6,
                         "Mnnz_per_s": p.nnz / (mean * 1e-3) / 1e6,
                         "algorithmic_bytes": abytes, "GBps": abytes / (mean * 1e-3) / 1e9,
                         "hbm_frac": abytes / (mean * 1e-3) / 1e9 / hbm_peak, "value_bytes": p.nnz * sT}
        forms[f"k{k}"] = res
        del p, vals, q, me
    forms["f64"] = {"value": forms["k2"]["f64"]["Mnodes_per_s"]}
    return dict(forms=forms, metric="3D P_k mass (App. D), k = 1..6 at about 10^6 nodes: M nodes/s, fixed "
                                    "pattern (value: k = 2, FP64)", unit="M nodes/s",
                config={"workload": "Kuhn cube, P_k lattice nodes, kN ~ 100 (about 1.03e6 nodes), jitter 0.15h, "
                                    "elements permuted", "hbm_peak_GBps": hbm_peak})


def wl_boundary(fe, torch, K, W, flush, hbm_peak, N=2000):
    """Facet mass and P1-weighted mass of an 8M-triangle surface in 3D, as generated and Morton-renumbered."""
    from paper_1401_3301_gb300 import meshgen
    forms = {}
    # facet (boundary) mass and P1-weighted mass on a large triangulated surface in 3D,
    # as generated (random vertex numbering) and after fe_morton_vertex_order
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
        for name, prec, T in _forms(fe, torch):
            vals = torch.empty(p.nnz, dtype=T, device="cuda")
            w = wv.to(T)
            res = {}
            for label, fn in (("mass", lambda: fe.fe_assemble_mass(p, q, prec=prec, vals=vals)),
                              ("wmass_p1", lambda: fe.fe_assemble_wmass(p, q, w, fe.COEF_P1, prec=prec,
                                                                        vals=vals))):
                med, mean = _timed(fn, K, W, flush)
                p.check()
                res[label] = {"ms_per_step": mean, "ms_median": med, "value": m.nme / (mean * 1e-3) / 1e6}
            forms.setdefault(name, {"value": None, "numbering": {}})["numbering"][label_n] = res
        nnz = p.nnz
        del p
    for name in ("f64", "f32", "f64x"):
        forms[name]["value"] = forms[name]["numbering"]["morton"]["mass"]["value"]
    return dict(forms=forms, metric="3D surface (facet) mass and P1-weighted mass, Mtris/s, fixed pattern "
                                    "(value: Morton vertex numbering, mass)", unit="Mtris/s",
                config={"workload": f"height-field surface over the unit square, N={N} ({m.nme:,} triangles, "
                                    f"{m.nq:,} vertices), jitter 0.2h, vertices and elements permuted",
                        "nnz": nnz, "pattern_build_ms": pms})


# the default run prints these beside the headline (shorter runs); --workload X prints one
SECONDARY = {"mass": wl_mass, "elas": wl_elas, "2d": wl_2d, "batched": wl_batched, "diff": wl_diff}
ALL_WORKLOADS = {**SECONDARY, "general": wl_general, "pk": wl_pk, "boundary": wl_boundary}


def run_other(args):
    import torch
    from paper_1401_3301_gb300 import build_ext, fe
    build_ext.build()
    fe.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hbm_peak, _, _ = measured_peaks()
    name = "mass" if args.workload in ("mass", "wmass") else args.workload
    extra = {"count": args.batch_meshes, "replays": args.replays} if name == "batched" else {}
    res = ALL_WORKLOADS[name](fe, torch, args.steps, args.warmup, flush, hbm_peak, **extra)
    outs = res.values() if name == "mass" else [res]
    for out in outs:
        line = {"workload": name, "data": "synthetic", "steps": args.steps, "warmup": args.warmup, "n_gpus": 1,
                "higher_is_better": True, **out}
        line["value"] = out["forms"]["f64"]["value"]
        line["dtype"] = "f64"
        print(json.dumps(line), flush=True)


def secondary_workloads(fe, torch, flush, hbm_peak, steps=20, warmup=3):
    """The other configurations of the hot path, measured compactly for the headline line:
    per workload and form the throughput, step time, per-kernel times and the dominant
    kernel's HBM fraction."""
    out = {}
    for name, fn in SECONDARY.items():
        try:
            r = fn(fe, torch, steps, warmup, flush, hbm_peak)
        except Exception as e:  # noqa: BLE001 - a failed secondary workload must not lose the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}
            continue
        for key, val in (r.items() if name == "mass" else [(name, r)]):
            out[key] = val
        torch.cuda.empty_cache()
    return out


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

#!/usr/bin/env python
"""Benchmark of the Kirchhoff network solve on one GB300 (or N, one per rank).

One step = the whole hot path on one 2048 x 2048 network with long-range
correlated conductances (FBM, H = 0.7, sigma = 1.5; seeded, synthetic):
net_create on device-resident bond planes (packing, cluster labelling,
Jacobi scaling), the mixed-precision solve (FP32 CG inside FP64 iterative
refinement to a 1e-11 relative residual), and the face flows.  The value is
solves per second over all ranks (each rank solves its own instance: weak
scaling, no collective on the data path).  The FP64 CG on the same network is
timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Solves/s & p99 latency; CG HBM GB/s; mixed vs FP64 CG at 1e-8 rel. conductance"
WORKLOAD = "2D 2048x2048 bond network, FBM H=0.7 sigma=1.5 conductances, K_x"
TOL_REL = 1e-11
L2_FLUSH_BYTES = 512 << 20


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the 256^3 percolation, batch and serve "
                         "measurements that the default run adds to its line")
    ap.add_argument("--workload", default="fbm2048",
                    choices=["fbm2048", "perc3d", "batch", "serve", "aniso", "periodic", "corrperc",
                             "fbmgen"],
                    help="fbm2048: the headline 2048^2 solve; perc3d: 256^3 percolation; batch: "
                         "512 networks in one batched solve; serve: the request queue; aniso: "
                         "K_x/K_y of anisotropic FBM networks (both axes batched)")
    ap.add_argument("--fbm-log2", default="24,28,30",
                    help="fbmgen: log2 of the node counts (even), comma separated")
    ap.add_argument("--aniso-size", type=int, default=512)
    ap.add_argument("--aniso-real", type=int, default=8)
    ap.add_argument("--aniso-bc", default="periodic", choices=["periodic", "noflow"],
                    help="aniso: transverse faces periodic (the paper's, Sec. II; K_y from the "
                         "transposed field) or no-flow")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--fp64", action="store_true",
                    help="with --profile-solve: an FP64 inner loop instead of FP32")
    ap.add_argument("--profile-solve", action="store_true",
                    help="one set-up and one refinement step on the workload, printing the inner "
                         "iteration count (for normalising profiler counters per iteration)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """Hash of the persistent kernel's code (its source and headers with
    // comments and blank lines left out: the counters depend on the code)."""
    h = hashlib.sha256()
    for name in ("cg_persist.cu", "common.cuh", "ffloat.cuh", "tma.cuh"):
        for line in open(os.path.join(ROOT, "paper_1908_03301_gb300", "csrc", name), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel_hash):
    """DRAM bytes per CG iteration of the inner kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "cg_persist_fbm2048.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_iteration")


def measured_hbm_peak():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else
    the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_oracle(name):
    p = os.path.join(ROOT, "tests", "golden", "oracle_full_size.json")
    if not os.path.exists(p):
        return None
    return json.load(open(p)).get(name)


def oracle_sample(dims, planes, seconds=15.0, nthreads=0):
    """Time the oracle's Jacobi-PCG on the full network for a bounded number of
    iterations (nthreads = 0: all cores); returns (seconds per iteration,
    set-up seconds, iterations run, threads)."""
    import oracle

    it = 8
    t = time.perf_counter()
    oracle.solve(dims, planes, max_iter=1, tol=0.0, nthreads=nthreads)  # set-up (labels, diagonal)
    t_setup = time.perf_counter() - t
    while True:
        t = time.perf_counter()
        oracle.solve(dims, planes, max_iter=it, tol=0.0, nthreads=nthreads)
        dt = time.perf_counter() - t
        if dt > seconds / 3 or it >= 4096:
            break
        it *= 2
    per_it = max(dt - t_setup, 1e-9) / (it - 1)
    return per_it, t_setup, it, (nthreads if nthreads > 0 else oracle.max_threads())


# ---------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    if rank != 0:
        return
    from paper_1908_03301_gb300 import netgen

    dims, planes = netgen.workload_fbm2d(n=a.size)
    ref = stored_oracle("fbm2048_iso_x") if a.size == 2048 else None
    iters = ref["iters"] if ref else None
    step_s = []
    for k in range(a.warmup + a.steps):
        per_it, t_setup, it, th = oracle_sample(dims, planes, seconds=6.0)
        if k >= a.warmup:
            step_s.append(t_setup + per_it * (iters or 1))
    mean_s = statistics.mean(step_s)
    val = 1.0 / mean_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": mean_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": dims[0] * dims[1], "tol_rel": 1e-13,
                       "solver": "FP64 Jacobi-PCG CPU oracle"},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": th, "kind": "oracle",
                             "sample": f"{it} oracle CG iterations on the full network per step, "
                                       f"scaled to the {iters} iterations of its full solve "
                                       f"(stored by tests/golden/make_oracle_reference.py)"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(a, rank, world, local):
    import numpy as np
    import torch

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ns.lib(build_if_missing=(world == 1))
    seed = netgen.SEED_BASE + 1 if rank == 0 else netgen.SEED_BASE + 1000 * 1 + rank
    dims, planes = netgen.workload_fbm2d(n=a.size, seed=seed)
    tplanes = [torch.from_numpy(g).to(dev) for g in planes]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(precision):
        net = ns.Network(dims, tplanes)
        r = net.solve(ns.make_opts(precision=precision, tol_rel=TOL_REL,
                                   stream=stream.cuda_stream))
        q = net.flux()
        net.close()
        return r, q

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(precision, steps, warmup):
        for _ in range(warmup):
            step(precision)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = []
        res = []
        t0 = time.perf_counter()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r, q = step(precision)
            e1.record(stream)
            evs.append((e0, e1))
            res.append(r)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        return ms, res, wall

    with Clocks(local) as clk:
        ms, res, wall = timed(ns.NET_MIXED, a.steps, a.warmup)
    clocks = clk.summary()
    total_ms = sum(ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * a.steps / (total_ms / 1e3)

    # FP64 CG comparator on the same network
    ms64, res64 = [], []
    if a.fp64_steps > 0:
        ms64, res64, _ = timed(ns.NET_FP64, a.fp64_steps, 1)

    # end to end through the public API from pinned host memory
    pinned = [torch.from_numpy(g).pin_memory() for g in planes]
    hplanes = [p.numpy() for p in pinned]
    N = dims[0] * dims[1]
    Pout = torch.empty(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e_t = []
    for k in range((1 + a.e2e_steps) if a.e2e_steps > 0 else 0):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        net = ns.Network(dims, hplanes)
        r = net.solve(ns.make_opts(tol_rel=TOL_REL))
        lib = ns.lib()
        st = lib.net_get_pressure(net.h, Pout.data_ptr(), N, 0)
        net.close()
        dt = time.perf_counter() - t
        assert st == 0
        if k > 0:
            e2e_t.append(dt)
    h2d = sum(g.nbytes for g in planes)
    d2h = N * 8 + 64

    if rank != 0:
        return
    r0 = res[-1]
    d = len(dims)
    b_alg = 32 + 4 * d  # bytes per active unknown per FP32 inner iteration
    inner_s = r0.inner_ms / 1e3
    achieved = b_alg * r0.n_active * r0.inner_iters / inner_s / 1e9 if inner_s > 0 else None
    peak, peak_src = measured_hbm_peak()
    khash = kernel_source_hash()
    traffic = profiled_traffic(khash)
    dram_gbs = traffic * r0.inner_iters / inner_s / 1e9 if (traffic and inner_s > 0) else None
    ref = stored_oracle("fbm2048_iso_x") if a.size == 2048 else None
    rel_vs_oracle = abs(r0.g_eff - ref["g_eff"]) / ref["g_eff"] if ref else None
    rel64 = abs(res64[-1].g_eff - ref["g_eff"]) / ref["g_eff"] if (ref and res64) else None
    launches_setup = d + 5 + 1 + 1
    launches = launches_setup + 1 + (1 + r0.outer_iters) + r0.inner_launches
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": N, "n_active": r0.n_active,
                   "precision": "FP32 inner CG / FP64 refinement", "tol_rel": TOL_REL,
                   "l2": "flushed between steps (512 MiB write)"},
        "p50_ms": statistics.median(ms),
        "p99_ms": float(np.percentile(ms, 99)),
        "wall_s": wall,
        "accuracy": {"g_eff": r0.g_eff, "rel_err_vs_oracle": rel_vs_oracle,
                     "rel_residual": r0.rel_residual, "max_imbalance": r0.max_imbalance,
                     "outer_iters": r0.outer_iters, "inner_iters": r0.inner_iters,
                     "fp64_fallback": r0.fp64_fallback},
        "fp64_cg": ({"value": a.fp64_steps / (sum(ms64) / 1e3), "unit": "solves/s",
                     "ms_per_step": statistics.mean(ms64), "inner_iters": res64[-1].inner_iters,
                     "g_eff": res64[-1].g_eff, "rel_err_vs_oracle": rel64,
                     "speedup_mixed_over_fp64": statistics.mean(ms64) / statistics.mean(ms)}
                    if ms64 else None),
        "cg_algorithmic_gbs": achieved,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "cg_persist_kernel (one CG iteration = one unit)",
                     "peak_source": peak_src, "bytes_per_unknown_iter": b_alg,
                     "algorithmic_bytes_per_iteration": b_alg * r0.n_active,
                     "dram_gbs": dram_gbs, "dram_frac": (dram_gbs / peak) if dram_gbs else None,
                     "note": "achieved = algorithmic bytes (40 B x unknowns) per iteration / time per "
                             "iteration; y, r, p and q stay in an L2 set-aside during the solve, so "
                             "DRAM carries only `traffic` bytes per iteration (ncu, same kernel "
                             "source): dram_gbs = traffic / time per iteration"},
        "e2e": ({"value": len(e2e_t) / sum(e2e_t), "unit": "solves/s",
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h} if e2e_t else None),
        "gpu_launches": int(launches * a.steps),
        "clocks": clocks,
    }
    if world == 1 and not a.no_extra:
        # the other workloads, each under its own clock record
        line["configs"] = {}
        for name, fn in (("perc3d", lambda: perc3d_line(a, 3, 1, 1)),
                         ("batch", lambda: batch_line(a, 0, 1, local, 1, 1)),
                         ("serve", lambda: serve_line(a, 400, (0.5,), 150))):
            t = time.perf_counter()
            try:
                sub = fn()
            except Exception as e:  # reported, the headline stands
                sub = {"error": f"{type(e).__name__}: {e}"}
            if isinstance(sub, dict):
                sub.pop("metric", None)
                sub["bench_wall_s"] = time.perf_counter() - t
            line["configs"][name] = sub
    if world == 1 and not a.no_cpu_baseline:
        it_full = ref["iters"] if ref else None
        per_it, t_setup, it, th = oracle_sample(dims, planes, seconds=15.0)
        if it_full:
            v = 1.0 / (t_setup + per_it * it_full)
            sample = (f"{it} oracle CG iterations on the full 2048^2 network, scaled to the "
                      f"{it_full} iterations of its full solve")
            line["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": th, "kind": "oracle",
                                    "sample": sample}
        else:
            line["cpu_baseline"] = {"value": 1.0 / per_it / 1.0, "unit": "CG iterations/s",
                                    "cores": th, "kind": "oracle",
                                    "sample": f"{it} oracle CG iterations on the full network"}
        if it_full:
            # the same on one thread (then every later oracle call names its threads)
            per1, setup1, it1, _ = oracle_sample(dims, planes, seconds=12.0, nthreads=1)
            line["cpu_baseline"]["one_thread"] = {
                "value": 1.0 / (setup1 + per1 * it_full), "unit": "solves/s", "cores": 1,
                "sample": f"{it1} oracle CG iterations on one thread, scaled to {it_full}"}
        line["cpu_baseline"]["full_solve_64x64"] = oracle_full_small(th)
    print(json.dumps(line), flush=True)


def oracle_full_small(threads_all):
    """One full oracle solve of the 64 x 64 workload (g = 10^U(-1,1)) to a
    1e-12 relative residual, wall-clock, on one thread and on all cores."""
    import oracle
    from paper_1908_03301_gb300 import netgen

    dims, planes, _ = netgen.workload_small("random")
    out = {"workload": "2D 64x64, g=10^U(-1,1), tol 1e-12", "cores": threads_all}
    for key, nth in (("one_thread_s", 1), ("all_cores_s", threads_all)):
        best = None
        for _ in range(5):
            t = time.perf_counter()
            r = oracle.solve(dims, planes, tol=1e-12, nthreads=nth)
            dt = time.perf_counter() - t
            best = dt if best is None else min(best, dt)
        out[key] = best
        out["iters"] = r.iters
    return out


def run_profile_solve(a):
    """One net_create + one refinement step (one inner CG solve).  --workload
    perc3d profiles an n^3 percolation network of the 256^3 workload's kind
    (n = --size), anything else an n^2 FBM network."""
    import torch

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    if a.workload == "perc3d":
        dims, planes = netgen.workload_perc3d(n=a.size)
    else:
        dims, planes = netgen.workload_fbm2d(n=a.size)
    tplanes = [torch.from_numpy(g).cuda() for g in planes]
    net = ns.Network(dims, tplanes)
    prec = ns.NET_FP64 if a.fp64 else ns.NET_MIXED
    r = net.solve(ns.make_opts(precision=prec, max_outer=1, tol_rel=TOL_REL), check=False)
    net.close()
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": True, "fp64": a.fp64, "dims": list(dims), "inner_iters": r.inner_iters,
                      "inner_ms": r.inner_ms, "n_active": r.n_active, "n_solved": r.n_solved,
                      "inner_launches": r.inner_launches}), flush=True)


# ---------------------------------------------------------------- other workloads
def _clocked(fn):
    with Clocks(0) as clk:
        out = fn()
    return out, clk.summary()


def run_perc3d(a):
    print(json.dumps(perc3d_line(a, a.steps, a.warmup, max(1, a.fp64_steps))), flush=True)


def perc3d_line(a, n_steps, n_warmup, n_fp64):
    """256^3 bond percolation (p = 0.26, FP32 conductances from a 3D FBM):
    labelling + mixed solve per step, FP64 solve beside it."""
    import torch

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    dims, planes = netgen.workload_perc3d()
    dev = torch.device("cuda", 0)
    tplanes = [torch.from_numpy(g).to(dev) for g in planes]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def steps(precision, k, w):
        for _ in range(w):
            with ns.Network(dims, tplanes) as net:
                net.solve(ns.make_opts(precision=precision, tol_rel=TOL_REL, stream=stream.cuda_stream))
        ms, res = [], []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with ns.Network(dims, tplanes) as net:
                r = net.solve(ns.make_opts(precision=precision, tol_rel=TOL_REL, stream=stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            res.append(r)
        return ms, res

    (ms, res), clocks = _clocked(lambda: steps(ns.NET_MIXED, n_steps, n_warmup))
    ms64, res64 = steps(ns.NET_FP64, n_fp64, 1)
    r0 = res[-1]
    N = dims[0] * dims[1] * dims[2]
    b_alg = 44 * r0.n_solved  # 32 + 4d bytes per unknown of the linear system
    it_s = r0.inner_ms / 1e3 / max(1, r0.inner_iters)
    peak = measured_hbm_peak()[0]
    # one launch per inner solve: the compacted solve; otherwise lattice sweeps
    compact = r0.inner_launches <= 2 * max(1, r0.outer_iters)
    ref = stored_oracle("perc256_x")
    line = {"metric": METRIC, "workload": "perc3d", "value": len(ms) / (sum(ms) / 1e3),
            "unit": "solves/s", "ms_per_step": statistics.mean(ms), "p50_ms": statistics.median(ms),
            "steps": len(ms), "warmup": n_warmup, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "3D 256^3 bond percolation p=0.26, FBM H=0.3 sigma=1, FP32 "
                                   "conductances", "nodes": N, "n_active": r0.n_active,
                       "n_solved": r0.n_solved, "tol_rel": TOL_REL},
            "accuracy": {"g_eff": r0.g_eff, "g_eff_fp64": res64[-1].g_eff,
                         "rel_mixed_vs_fp64": abs(r0.g_eff - res64[-1].g_eff) / max(abs(res64[-1].g_eff), 1e-300),
                         "rel_err_vs_oracle": (abs(r0.g_eff - ref["g_eff"]) / ref["g_eff"]) if ref else None,
                         "rel_residual": r0.rel_residual, "max_imbalance": r0.max_imbalance,
                         "outer_iters": r0.outer_iters, "inner_iters": r0.inner_iters,
                         "fp64_fallback": r0.fp64_fallback},
            "fp64_cg": {"value": len(ms64) / (sum(ms64) / 1e3), "unit": "solves/s",
                        "ms_per_step": statistics.mean(ms64), "inner_iters": res64[-1].inner_iters,
                        "speedup_mixed_over_fp64": statistics.mean(ms64) / statistics.mean(ms)},
            "roofline": {"bound": "hbm", "kernel": "compact_cg_kernel (listed unknowns)" if compact
                         else "sweep_kernel (lattice)",
                         "us_per_iteration": it_s * 1e6,
                         "achieved": b_alg / it_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": b_alg / it_s / 1e9 / peak,
                         "unknown_iterations_per_s": r0.n_solved / it_s,
                         "bytes_note": "achieved = 44 B x unknowns of the linear system (after cluster "
                                       "stripping and removal of dead-end trees and loops) per CG "
                                       "iteration / inner-loop time per iteration; peak = measured copy"},
            "clocks": clocks}
    return line


def run_batch(a, rank=0, world=1, local=0):
    line = batch_line(a, rank, world, local, a.steps, a.warmup)
    if line is not None:
        print(json.dumps(line), flush=True)


def batch_line(a, rank, world, local, n_steps, n_warmup):
    """512 independent 2D networks (sides 64..1024, lognormal sigma=1, even
    ones percolated at p=0.55) created and solved together per step.  Under
    torchrun the networks are shared out over the ranks (longest first by
    estimated work, no data-path collective); the step time is the max over
    ranks, so the value is strong-scaling throughput of the fixed set."""
    import torch

    from paper_1908_03301_gb300 import netgen, replicas
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=(world == 1))
    all_dims = [netgen.batch_instance_dims(i) for i in range(a.batch_count)]
    mine = replicas.my_share(all_dims, rank, world)
    specs = [netgen.batch_instance(i) for i in mine]
    dev = torch.device("cuda", local)
    tpl = [[torch.from_numpy(g).to(dev) for g in planes] for _, planes in specs]
    nodes = sum(d[0] * d[1] for d in all_dims)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    split = []  # (set-up seconds, solve seconds) of each step

    def one():
        t0 = time.perf_counter()
        nets = [ns.Network(d, t) for (d, _), t in zip(specs, tpl)]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        res = ns.solve_batch(nets, ns.make_opts(tol_rel=TOL_REL))
        split.append((t1 - t0, time.perf_counter() - t1))
        for n in nets:
            n.close()
        return res

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(n_warmup):
        one()
    torch.cuda.synchronize()
    barrier()
    times, res = [], None
    with Clocks(local) as clk:
        for _ in range(n_steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            t = time.perf_counter()
            res = one()
            torch.cuda.synchronize()
            times.append(replicas.max_over_ranks(time.perf_counter() - t, device=dev))
    clocks = clk.summary()
    local_res = {i: (r.status, r.inner_iters * r.n_solved, r.ms, r.fp64_fallback,
                     r.inner_iters * specs[k][0][0] * specs[k][0][1], r.g_eff_err)
                 for k, (i, r) in enumerate(zip(mine, res))}
    allr = replicas.gather_results(local_res, a.batch_count)
    if rank != 0:
        return None
    ui = sum(x[1] for x in allr)
    li = sum(x[4] for x in allr)
    setup_s = statistics.mean(x[0] for x in split[-len(times):])
    solve_s = statistics.mean(x[1] for x in split[-len(times):])
    ok = sum(x[0] == 0 for x in allr)
    lat = sorted(x[2] for x in allr)
    peak = measured_hbm_peak()[0]
    alg = 40 * ui / statistics.mean(times) / 1e9
    line = {"metric": METRIC, "workload": "batch", "value": a.batch_count * len(times) / sum(times),
            "unit": "solves/s", "n_gpus": world, "ms_per_step": statistics.mean(times) * 1e3,
            "steps": len(times), "warmup": n_warmup, "scaling": "strong", "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{a.batch_count} 2D networks, sides U{{64..1024}}, lognormal "
                                   "sigma=1, even ones percolated p=0.55; created + net_solve_batch",
                       "nodes": nodes, "tol_rel": TOL_REL,
                       "parallelism": f"networks sharded over {world} GPU(s), no collective"},
            "converged": ok, "unknown_iterations_per_s": ui / statistics.mean(times),
            "algorithmic_gbs": alg,
            "lattice_gbs": 40 * li / statistics.mean(times) / 1e9,
            "roofline": {"bound": "hbm", "kernel": "sweep_kernel (all running networks per launch)",
                         "achieved": alg, "peak": peak, "unit": "GB/s", "frac": alg / peak,
                         "lattice_frac": 40 * li / statistics.mean(times) / 1e9 / peak,
                         "solve_only_frac": 40 * ui / solve_s / 1e9 / peak,
                         "solve_only_lattice_frac": 40 * li / solve_s / 1e9 / peak,
                         "note": "achieved / frac: whole-batch wall time including the set-up of "
                                 "every network; solve_only: net_solve_batch alone; 40 B per unknown "
                                 "of each linear system (lattice: per lattice node) per CG iteration"},
            "setup_s": setup_s, "solve_s": solve_s,
            "accuracy": {"max_g_eff_err_estimate": max(x[5] for x in allr)},
            "bytes_note": "algorithmic = 40 B x unknowns in the linear system (dead ends and "
                          "non-spanning clusters excluded) x CG iterations; lattice = 40 B x "
                          "all lattice nodes x CG iterations (what the sweep streams)",
            "per_network_ms_p50": lat[len(lat) // 2], "per_network_ms_p99": lat[int(0.99 * (len(lat) - 1))],
            "fp64_fallbacks": sum(x[3] for x in allr), "clocks": clocks}
    return line


def run_serve(a):
    print(json.dumps(serve_line(a, a.serve_requests, (0.25, 0.5, 0.8), max(32, a.serve_requests // 2))),
          flush=True)


def serve_line(a, n_sat, fracs, n_sweep):
    """Poisson request stream of mixed networks (70 % 2D sides 32..1024, 30 %
    3D sides 16..128; FBM or lognormal; 20 % near-critical percolation)
    through the queue with a 150 GB budget.  n_sat distinct requests (fresh
    seeded draws, generated up front) arrive at --serve-rate (saturation);
    then, for each fraction in fracs, the first n_sweep of them at that
    fraction of the measured capacity.  Per-request accuracy: the solver's
    first-order estimate of the relative G_eff error, maximum over requests."""
    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    t = time.perf_counter()
    pool = [netgen.request_instance(i) for i in range(max(n_sat, n_sweep, 16))]
    gen_s = time.perf_counter() - t

    def run(rate, n):
        arr = netgen.poisson_arrivals(n, rate)
        with ns.Queue(mem_budget_bytes=150 << 30, max_slots=256, opts=ns.make_opts(tol_rel=TOL_REL)) as q:
            tickets = []
            t0 = time.perf_counter()
            for i in range(n):
                dt = arr[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                d, pl = pool[i]
                tickets.append(q.submit(d, pl))
            results = [q.wait(t, timeout_ms=600000) for t in tickets]
            t1 = time.perf_counter()
            p50, p99, done = q.stats()
        ok = sum(st == 0 for st, _ in results)
        counts = {}
        for st, _ in results:
            name = ns.STATUS_NAMES[st] if 0 <= st < len(ns.STATUS_NAMES) else str(st)
            counts[name] = counts.get(name, 0) + 1
        errors = sorted({r.error for st, r in results if st != 0 and r is not None})[:4]
        worst = max((r.g_eff_err for st, r in results if st == 0 and r is not None), default=None)
        waits = sorted(r.queue_ms for st, r in results if r is not None)
        beside = sum(1 for st, r in results if r is not None and r.co_running > 0)

        def pct(v, f):
            return v[min(len(v) - 1, int(f * (len(v) - 1) + 0.5))] if v else None

        return {"offered_rate": rate, "requests": n, "ok": ok, "status_counts": counts, "errors": errors,
                "solves_per_s": n / (t1 - t0), "p50_ms": p50, "p99_ms": p99, "wall_s": t1 - t0,
                "queue_wait_p50_ms": pct(waits, 0.5), "queue_wait_p99_ms": pct(waits, 0.99),
                "admitted_beside_running": beside, "max_g_eff_err_estimate": worst}

    run(50.0, 16)  # warm-up
    with Clocks(0) as clk:
        sat = run(a.serve_rate, n_sat)
    clocks = clk.summary()
    cap = sat["solves_per_s"]
    sweep = [run(f * cap, n_sweep) for f in fracs]
    line = {"metric": METRIC, "workload": "serve", "value": sat["solves_per_s"], "unit": "solves/s",
            "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"], "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"Poisson stream at {a.serve_rate:g}/s, 70% 2D (32..1024) / 30% 3D "
                                   f"(16..128), FBM or lognormal, 20% near-critical percolation, 150 GB "
                                   f"budget; {n_sat} distinct requests (seeded draws)",
                       "tol_rel": TOL_REL, "generation_s": gen_s},
            "latency_note": "p50/p99 from arrival to result; at saturation they are dominated by "
                            "queueing (the offered rate is above capacity), the sweep gives service "
                            "latency below capacity",
            "saturated": sat, "sweep": sweep, "clocks": clocks}
    return line


def run_aniso(a):
    """Permeability anisotropy K_x/K_y (Sec. VI.B, Fig. 10): for H in {0.75,
    0.35} and beta_x/beta_y in {0.2, 0.5, 1, 2, 5}, --aniso-real realizations
    of an n x n anisotropic FBM network (Eq. 2, sigma = 1), each solved along x
    and along y; every (H, ratio) is one net_solve_batch of 2 x realizations.
    Reports min / median / max of K_x/K_y per cell and solves/s overall."""
    import numpy as np

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    n, R = a.aniso_size, a.aniso_real
    cells, total_s, solves, worst = [], 0.0, 0, 0.0
    per = a.aniso_bc == "periodic"
    for hi, H in enumerate(netgen.ANISO_H):
        for ri, ratio in enumerate(netgen.ANISO_RATIOS):
            if per:  # both axes as flow along x with periodic y: the field and its transpose
                nets = [ns.Network(d, p, periodic=(1,)) for r in range(R)
                        for d, p in netgen.aniso_pair_periodic(hi, ri, r, n=n)]
            else:
                specs = [netgen.aniso_instance(hi, ri, r, n=n) for r in range(R)]
                nets = [ns.Network(d, p, flow_axis=ax) for d, p in specs for ax in (0, 1)]
            t = time.perf_counter()
            res = ns.solve_batch(nets, ns.make_opts(tol_rel=TOL_REL))
            total_s += time.perf_counter() - t
            for net in nets:
                net.close()
            solves += len(res)
            assert all(x.status == 0 for x in res), [x.status for x in res]
            kx = np.array([res[2 * r].k_eff for r in range(R)])
            ky = np.array([res[2 * r + 1].k_eff for r in range(R)])
            worst = max(worst, max(x.g_eff_err for x in res))
            ratio_k = kx / ky
            cells.append({"H": H, "beta_x_over_beta_y": ratio, "kx_over_ky_min": float(ratio_k.min()),
                          "kx_over_ky_median": float(np.median(ratio_k)),
                          "kx_over_ky_max": float(ratio_k.max())})
    line = {"metric": METRIC, "workload": "aniso", "value": solves / total_s, "unit": "solves/s",
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{n}x{n} anisotropic FBM networks (Eq. 2), sigma=1, {R} realizations "
                                   "per (H, beta_x/beta_y), K_x and K_y batched; transverse faces "
                                   + ("periodic (K_y from the transposed field)" if per else "no-flow"),
                       "tol_rel": TOL_REL},
            "solves": solves, "seconds": total_s, "max_geff_err_estimate": worst, "cells": cells,
            "paper_ranges": {"H=0.75": [0.6, 1.6], "H=0.35": [0.5, 2.5],
                             "note": "Fig. 10 bounds (3.6M-node networks); context only"}}
    print(json.dumps(line), flush=True)


def run_periodic(a):
    """The 2048^2 FBM network of the headline (H = 0.7, sigma = 1.5) with the
    paper's own boundaries (Sec. II): pressure drop along x, periodic y.  The
    network is resident; each step is one mixed solve (L2 flushed before it).
    The persistent 2D kernel takes the wrap rows into its halo exchange; the
    FP64 comparator runs the compacted solve, whose neighbour table holds the
    wrap bonds.  The same network with no-flow y is the headline."""
    import torch

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    dims, planes = netgen.workload_fbm2d(periodic=(1,))
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    net = ns.Network(dims, planes, periodic=(1,))

    def steps(precision, k, w):
        opts = ns.make_opts(precision=precision, tol_rel=TOL_REL, stream=stream.cuda_stream)
        for _ in range(w):
            net.solve(opts)
        ms, res = [], []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = net.solve(opts)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            res.append(r)
        return ms, res

    (ms, res), clocks = _clocked(lambda: steps(ns.NET_MIXED, a.steps, a.warmup))
    ms64, res64 = steps(ns.NET_FP64, max(1, a.fp64_steps), 1)
    net.close()
    r0 = res[-1]
    b_alg = 40 * r0.n_solved  # 32 + 4d bytes per unknown and iteration, d = 2
    it_s = r0.inner_ms / 1e3 / max(1, r0.inner_iters)
    peak = measured_hbm_peak()[0]
    line = {"metric": METRIC, "workload": "periodic", "value": len(ms) / (sum(ms) / 1e3),
            "unit": "solves/s", "ms_per_step": statistics.mean(ms), "steps": len(ms),
            "warmup": a.warmup, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "2D 2048^2 FBM network H=0.7 sigma=1.5, flow along x, periodic y "
                                   "(network resident, L2 flushed between steps)",
                       "n_solved": r0.n_solved, "tol_rel": TOL_REL},
            "accuracy": {"g_eff": r0.g_eff, "g_eff_fp64": res64[-1].g_eff,
                         "rel_mixed_vs_fp64": abs(r0.g_eff - res64[-1].g_eff) / max(abs(res64[-1].g_eff), 1e-300),
                         "g_eff_err_estimate": r0.g_eff_err, "outer_iters": r0.outer_iters,
                         "inner_iters": r0.inner_iters, "fp64_fallback": r0.fp64_fallback},
            "fp64_cg": {"value": len(ms64) / (sum(ms64) / 1e3), "unit": "solves/s",
                        "ms_per_step": statistics.mean(ms64), "inner_iters": res64[-1].inner_iters},
            "inner": {"kernel": "cg_persist_kernel (periodic y: wrap rows in the halo exchange)",
                      "us_per_iteration": it_s * 1e6, "algorithmic_gbs": b_alg / it_s / 1e9,
                      "frac": b_alg / it_s / 1e9 / peak,
                      "bytes_note": "algorithmic = 40 B x unknowns per CG iteration; peak = measured copy"},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_corrperc(a):
    """Correlated percolation by sorted removal (Sec. VI.B, Fig. 9): a
    1900^2 (3.6 M node) FBM network (H = 0.7, sigma = 1.5); for each q the
    fraction q of weakest bonds is closed on the device (net_close_smallest),
    then the network is created and solved.  Removing the weakest bonds of a
    correlated field cuts the network long before q = 1/2 (the threshold of
    uncorrelated bond percolation on this lattice): this realization spans up
    to q = 0.35 and not from q = 0.37, and the solve slows down on the way
    (critical slowing down).  Reports, per q, the removal time and its HBM
    rate, the solve time and iterations."""
    import torch

    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    dims = (1900, 1900)
    gen = netgen.rng(netgen.SEED_BASE + 6)
    host = netgen.fbm_bonds(dims, 0.7, 1.5, gen)
    dev = torch.device("cuda", 0)
    base = [torch.from_numpy(g).to(dev) for g in host]
    stream = torch.cuda.current_stream(dev)
    M = sum(g.numel() for g in base)
    cells, solve_ms = [], []
    for q in (0.1, 0.2, 0.3, 0.35, 0.4):
        rm, sv, res = [], [], None
        for it in range(a.warmup + a.steps):
            planes = [g.clone() for g in base]
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            ns.close_smallest(dims, planes, q)
            e[1].record(stream)
            with ns.Network(dims, planes) as net:
                r = net.solve(ns.make_opts(tol_rel=TOL_REL, stream=stream.cuda_stream))
            e[2].record(stream)
            torch.cuda.synchronize()
            if it >= a.warmup:
                rm.append(e[0].elapsed_time(e[1]))
                sv.append(e[1].elapsed_time(e[2]))
                res = r
        # 8 histogram passes over the FP64 bonds, one closing pass (read +
        # write of the closed ones): the algorithmic bytes of one removal
        b_rm = 9 * 8 * M + 8 * int(q * M)
        cells.append({"q": q, "removal_ms": statistics.mean(rm),
                      "removal_gbs": b_rm / (statistics.mean(rm) / 1e3) / 1e9,
                      "create_and_solve_ms": statistics.mean(sv), "g_eff": res.g_eff,
                      "n_active": res.n_active, "n_solved": res.n_solved,
                      "inner_iters": res.inner_iters, "status": res.status})
        solve_ms += [x + y for x, y in zip(rm, sv)]
    line = {"metric": METRIC, "workload": "corrperc", "value": len(solve_ms) / (sum(solve_ms) / 1e3),
            "unit": "solves/s", "steps": a.steps, "warmup": a.warmup, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "2D 1900^2 FBM network H=0.7 sigma=1.5, the weakest fraction q of "
                                   "bonds closed on the device, then created and solved; q in "
                                   "{0.1, 0.2, 0.3, 0.35, 0.4}", "bonds": M, "tol_rel": TOL_REL},
            "cells": cells}
    print(json.dumps(line), flush=True)


def run_fbmgen(a):
    """The FBM generator (Eq. 1) at the array sizes of the paper's Table I
    (2^24, 2^28 and 2^30 nodes: 4096^2, 16384^2, 32768^2), H = 0.7: noise ->
    filter -> inverse FFT -> normalised field -> FP32 conductance planes
    (sigma = 1.5), all on the device, with the FP32 transform (the value) and
    the FP64 one beside it.  The complex noise is drawn on the device before
    the timed region (the random draws are the generator's input); the draw's
    own time (torch's generator) is reported beside it, since Table I's times
    (MPI on four processes, context only) include their random draws."""
    import torch

    from paper_1908_03301_gb300 import netsolve as ns

    ns.lib(build_if_missing=True)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    paper_mpi_s = {24: 0.4, 28: 2.7, 30: 20.6}
    rows = []
    for lg in [int(v) for v in a.fbm_log2.split(",")]:
        n = 1 << (lg // 2)
        dims = (n, n)
        gen = torch.Generator(device=dev).manual_seed(netgen_seed(7) + lg)
        field = torch.empty((n, n), dtype=torch.float64, device=dev)
        row = {"nodes": n * n, "log2_nodes": lg, "paper_table1_mpi_s": paper_mpi_s.get(lg)}
        for tag, cdt in (("fft_f32", torch.complex64), ("fft_f64", torch.complex128)):
            ms_f, ms_b, ms_n = [], [], []
            for it in range(a.warmup + a.steps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[3].record(stream)
                noise = torch.randn((n, n), dtype=cdt, device=dev, generator=gen)
                e[0].record(stream)
                ns.fbm_field(dims, noise, 0.7, out=field)
                e[1].record(stream)
                planes = ns.fbm_bonds(dims, field, 1.5, torch.float32)
                e[2].record(stream)
                torch.cuda.synchronize()
                if it >= a.warmup:
                    ms_n.append(e[3].elapsed_time(e[0]))
                    ms_f.append(e[0].elapsed_time(e[1]))
                    ms_b.append(e[1].elapsed_time(e[2]))
                del noise, planes
            row[tag] = {"field_ms": statistics.mean(ms_f), "bonds_ms": statistics.mean(ms_b),
                        "total_ms": statistics.mean(ms_f) + statistics.mean(ms_b),
                        "noise_draw_ms_torch": statistics.mean(ms_n),
                        "field_check": {"mean": float(field.mean()), "var": float((field * field).mean())}}
        rows.append(row)
        del field
        torch.cuda.empty_cache()
    total = sum(r["fft_f32"]["total_ms"] for r in rows)
    line = {"metric": METRIC, "workload": "fbmgen", "value": len(rows) / (total / 1e3),
            "unit": "fields/s", "steps": a.steps, "warmup": a.warmup, "dtype": "f32 (FFT), f32 planes",
            "data": "synthetic",
            "config": {"workload": "2D FBM fields of 2^24, 2^28, 2^30 nodes, H=0.7, Eq. 1 spectral "
                                   "filtering + inverse FFT (cuFFT C2C FP32; Z2Z FP64 beside it) + "
                                   "normalisation, then FP32 conductance planes exp(1.5 (B_i+B_j)/2)"},
            "sizes": rows}
    print(json.dumps(line), flush=True)


def netgen_seed(k):
    from paper_1908_03301_gb300 import netgen

    return netgen.SEED_BASE + k


def main():
    a = args_()
    if a.profile_solve:
        run_profile_solve(a)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.workload in ("perc3d", "serve", "aniso", "periodic", "corrperc", "fbmgen") and a.impl == "ours":
        if rank == 0:
            {"perc3d": run_perc3d, "serve": run_serve, "aniso": run_aniso,
             "periodic": run_periodic, "corrperc": run_corrperc, "fbmgen": run_fbmgen}[a.workload](a)
        return
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        if a.workload == "batch":
            run_batch(a, rank, world, local)
        else:
            run_ours(a, rank, world, local)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

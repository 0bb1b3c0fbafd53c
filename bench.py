#!/usr/bin/env python
"""Benchmark of the collision-operator library on B300.

Workload (one "step"): the single-instance N = 128 configuration integrated in
full: build the kernel tensor for the grid (p/m in [1e-3, 10], m = 1), then
integrate the seeded bimodal f0 with the two freeze-in sources for the four
cross-sections sigma in {0.1, 1, 10, 100} (a batch of 4 instances sharing the
kernel) until each matches Maxwell-Boltzmann to 1e-3 in L1 after the sources
are off.  Metric: collision-term evaluations per second (C_proj for one
instance = one evaluation), with solves/s and the plain FP64 path on the same
inputs beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
(N > 1: launched by torch.distributed.run, one independent replica per rank.)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kx_inputs as ki  # noqa: E402

METRIC = "collision-term evals/s & solves/s vs plain FP64 path; p50/p99 solve latency"
UNIT = "evals/s"
L2_FLUSH_BYTES = 512 << 20     # > 126 MB L2
CSRC = os.path.join(ROOT, "paper_2607_00755_b300", "csrc")
# DRAM bytes (read + write) per launch from one-pass ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) of the named kernel, with the
# sha1 of the CUDA source file it was built from at capture time.  A capture
# is used only while the live kernel has the same name and algorithmic bytes
# and its source file is unchanged; otherwise the line's traffic is null and
# says why.
NCU_TRAFFIC = {
    "stream_n128_b1": {"kernel": "k_stream32r<1,2>", "stream_bytes": 6755176, "file": "kx_contract.cu",
                       "sha1": "7b419507fdaf8f1dd168de2e81803cfeecd4f506", "bytes": 6770688.0},
    "stream_n384": {"kernel": "k_stream32r<1,4>", "stream_bytes": 172449208, "file": "kx_contract.cu",
                    "sha1": "7b419507fdaf8f1dd168de2e81803cfeecd4f506", "bytes": 172477440.0 + 2772736.0},
    "stream_n512": {"kernel": "k_stream32r<1,4>", "stream_bytes": 406086712, "file": "kx_contract.cu",
                    "sha1": "7b419507fdaf8f1dd168de2e81803cfeecd4f506", "bytes": 406162432.0 + 2715136.0},
    "stage_n128_b1": {"kernel": "k_stage<1,0>", "stream_bytes": None, "file": "kx_contract.cu",
                      "sha1": "7b419507fdaf8f1dd168de2e81803cfeecd4f506", "bytes": 0.5 * (124416.0 + 128256.0)},
}


def source_sha1(name):
    import hashlib
    try:
        with open(os.path.join(CSRC, name), "rb") as fh:
            return hashlib.sha1(fh.read()).hexdigest()
    except OSError:
        return None


def traffic_for(key, kernel, stream_bytes=None):
    """(bytes per launch or None, note) for a kernel from its ncu capture."""
    cap = NCU_TRAFFIC.get(key)
    if not cap or cap["bytes"] is None:
        return None, "no ncu capture of this kernel"
    if not kernel.startswith(cap["kernel"]):
        return None, f"the capture is of {cap['kernel']}, the run uses {kernel}"
    if cap["stream_bytes"] is not None and stream_bytes is not None and cap["stream_bytes"] != stream_bytes:
        return None, "the kernel's tables changed since the capture"
    if source_sha1(cap["file"]) != cap["sha1"]:
        return None, f"{cap['file']} changed since the capture"
    return cap["bytes"], "one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum)"


def stream_kernel_name(ctx, n, batch):
    """Name of the FP32 streaming kernel the contraction of (n, batch) uses."""
    var, tuned = ctx.stream_variant(n, batch)
    vpl = 2 if n <= 160 else 4
    if var == 4:
        per = 1 if batch == 1 else (2 if batch == 2 else 4)
        return f"k_stream32p<{per},{vpl}> (whole share staged, {'tuned' if tuned else 'default rule'})"
    per = {0: 1, 1: 2, 2: 4, 3: 4}[var]
    name = f"k_stream32<4,4> (bulk-copy staged)" if var == 2 else f"k_stream32r<{per},{vpl}>"
    return f"{name} ({per} instance{'s' if per > 1 else ''} per pass, {'tuned' if tuned else 'default rule'})"


SOLVE = dict(t_end=1e5, h0=1e-3, rtol=1e-6, l1_tol=1e-3, check_every=10, max_attempts=2_000_000)
# FP64 operations the method does per grid point in one Heun stage (FMA = 2):
# C_raw = |M|^2 G (1), xi (1), the five projection moments (5 products, 5 sums),
# the correction xi (alpha + beta E) (2 FMA = 4), the sources (2 FMA = 4),
# k = C + S (1), and the update: stage 1 f + h k (2); stage 2 f + h/2 (k1 + k2)
# (3) and the error ratio |f_c - f_p| / (atol + rtol |f_c|) (4).
STAGE_FLOP_PER_POINT = {1: 23, 2: 28}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def workload():
    c = ki.config2()
    B = len(c["sigmas"])
    f0 = np.tile(c["f0"], (B, 1))
    atol = 1e-12 * float(c["f0"].max())
    return c, B, f0, dict(SOLVE, atol=atol)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(c, B, seconds: float):
    """The oracle as it stands: RHS evaluations (tensor-form C, projection,
    sources) of the workload's first Heun attempts, for about `seconds`."""
    import oracle
    q = c["q"]
    W = oracle.kernel_tensor(q)
    evals, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for b in range(B):
            M2 = oracle.M2_from_sigma(1.0, c["sigmas"][b])
            _, r = oracle.solve(q, W, c["f0"], M2, sources=c["sources"], t_end=1e5, h0=1e-3,
                                rtol=1e-6, atol=1e-12 * c["f0"].max(), max_attempts=2)
            evals += int(r["evals"])
    dt = time.perf_counter() - t0
    return evals, dt, oracle.num_threads()


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args, rank):
    """Reference arm: the FP64 CPU oracle on this host's cores (rank 0 only)."""
    if rank != 0:
        return 0
    c, B, f0, par = workload()
    per_step = max(1.0, min(8.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(c, B, per_step)
    tot_e, tot_t, cores = 0, 0.0, 1
    for _ in range(args.steps):
        e, t, cores = oracle_sample(c, B, per_step)
        tot_e += e
        tot_t += t
    val = tot_e / tot_t
    sample = (f"{tot_e} RHS evaluations (tensor-form C + projection + sources, first Heun "
              f"attempts of the 4-sigma N=128 workload) in {tot_t:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_desc(c, B),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_contraction_only(args):
    """Contraction kernel alone on an n-point grid (q in [1e-3, qmax]) for
    `batch` seeded bimodal distributions: cold L2 before every launch, or with
    --rotate R, R kernels of the grid whose contractions run back to back in
    rotation (each launch reads its tables from HBM when R x tables > L2)."""
    import torch
    import paper_2607_00755_b300 as kx
    ctx = kx.Context(0)
    q = ki.log_grid(args.n, 1e-3, args.qmax)
    prec = {"fp32": kx.FP32, "fp64": kx.FP64, "split": kx.SPLIT_TF32}[args.precision]
    ks = [ctx.build_kernel(q, precision=prec) for _ in range(max(1, args.rotate))]
    k = ks[0]
    f = torch.as_tensor(ki.batch_bimodal(np.random.default_rng(7), q, args.batch), device="cuda")
    if args.variant >= 0 and prec == kx.FP32:
        ctx.set_stream_variant(args.n, args.batch, args.variant)
    if args.rotate > 0:
        ms = ctx.time_contractions(ks, f, iters=args.iters, pdl=args.pdl)
    else:
        ms = ctx.time_contraction(k, f, iters=args.iters, flush_bytes=L2_FLUSH_BYTES)
    alg = k.info()["stream_bytes"]
    hbm, src = peaks()
    name = stream_kernel_name(ctx, args.n, args.batch) if prec == kx.FP32 else args.precision
    print(json.dumps({"kernel": "contraction", "variant": name, "n": args.n, "batch": args.batch,
                      "precision": args.precision, "rotate": args.rotate, "avg_ms": ms,
                      "algorithmic_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9,
                      "frac_of_" + src + "_hbm": alg / (ms * 1e-3) / 1e9 / hbm,
                      "info": k.info()}), flush=True)
    for kk in ks:
        kk.release()
    ctx.close()
    return 0


def tf32_peak():
    """TF32 dense peak: the measured bf16 figure times the nominal TF32/BF16
    ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal tf32/bf16"
    except Exception:
        return 1800.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16"


def measure_batched(ctx, kx, torch, flush, iters=5, check_sample=4):
    """Batched configuration: B = 512 seeded bimodal distributions sharing one
    N = 192 kernel (q in [1e-3, 1e2]); projected C per instance through
    kx_collision on the split-TF32 tensor-core path, with the exact loss and
    with the loss as a Chebyshev GEMM (K = 16), against the plain FP64 path on
    the same inputs.  Useful FLOP of one batch: the gain GEMM 2 P N B over the
    P = N (N + 1) / 2 symmetric pairs, and the Chebyshev loss GEMM 2 N (N K) B;
    split TF32 issues three products for each.  Returns the line and the first
    `check_sample` instances' outputs (compared with the FP64 oracle in the
    CPU-baseline leg)."""
    c = ki.config3()
    q, f, B = c["q"], c["f"], c["f"].shape[0]
    n = q.size
    stream = torch.cuda.current_stream()
    fd = torch.as_tensor(f, device="cuda")
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Cs = {}
    peak, peak_src = tf32_peak()
    # the raw tcgen05 kind::tf32 issue rate at this N tile (library microbenchmark),
    # at the SM clock's maximum, for context beside the contract's peak
    fpc, cyc = ctx.measure_mma_rate(0, n)
    mma_rate = fpc * 148 * 2.032e9 / 1e12
    P = n * (n + 1) // 2
    for name, prec, lt, reps, eta in (("split_tf32_exact_loss", kx.SPLIT_TF32, 0, iters, 0),
                                      ("split_tf32_cheb16_loss", kx.SPLIT_TF32, 16, iters, 0),
                                      ("split_tf32_bose_einstein", kx.SPLIT_TF32, 0, iters, 1),
                                      ("fp64", kx.FP64, 0, 2, 0)):
        k = ctx.build_kernel(q, precision=prec, loss_terms=lt, stats=eta)
        C, _ = ctx.collision(k, fd, c["sigma"])
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            e0.record(stream)
            C, _ = ctx.collision(k, fd, c["sigma"], out=C)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        Cs[name] = C[:check_sample].cpu().numpy()
        ms = tot / reps
        row = {"evals_per_s": B * reps / (tot / 1e3), "ms_per_batch": ms}
        if prec == kx.SPLIT_TF32:
            gain = 2.0 * P * n * B
            loss = 2.0 * n * (n * lt) * B if lt else 0.0
            useful = gain + loss
            row.update({"useful_gflop": useful / 1e9, "useful_tflops": useful / (ms * 1e-3) / 1e12,
                        "issued_tflops_split3": 3 * useful / (ms * 1e-3) / 1e12,
                        "frac_of_tf32_peak_issued": 3 * useful / (ms * 1e-3) / 1e12 / peak,
                        "tf32_peak_tflops": peak, "peak_source": peak_src,
                        "tf32_mma_issue_rate_tflops": mma_rate,
                        "frac_of_mma_issue_rate": 3 * useful / (ms * 1e-3) / 1e12 / mma_rate,
                        "mma_issue_rate_note": (f"tcgen05.mma kind::tf32 M=128 N={n} K=8 back to back from "
                                                f"shared memory: {cyc:.1f} cycles each, {fpc:.0f} FLOP/clk/SM, "
                                                "x 148 SMs x 2.032 GHz"),
                        "note": "whole kx_collision call (prep, both GEMMs or the exact loss, "
                                "row combine and projection), cold L2",
                        "launch_choices": ctx.split_tuning(k, B)})
        out[name] = row
        k.release()
    line = {"workload": "B=512 distributions sharing one N=192 kernel, q in [1e-3,1e2], "
                        "projected C (kx_collision)",
            "split_tf32": out["split_tf32_exact_loss"],
            "split_tf32_cheb16": out["split_tf32_cheb16_loss"],
            # the same batch with Bose-Einstein factors (eq. Lambda_quantum): the gain
            # GEMM and the exact loss kernel's three row sums
            "split_tf32_bose_einstein": out["split_tf32_bose_einstein"],
            "fp64_path": out["fp64"],
            "speedup_vs_fp64": out["split_tf32_exact_loss"]["evals_per_s"] / out["fp64"]["evals_per_s"],
            "speedup_vs_fp64_cheb16": out["split_tf32_cheb16_loss"]["evals_per_s"] / out["fp64"]["evals_per_s"],
            "max_rel_err_vs_oracle": None, "oracle_sample": f"{check_sample} instances"}
    check = {"q": q, "f": f[:check_sample], "sigma": c["sigma"][:check_sample], "C": Cs}
    return line, check


def measure_paper_runtime(ctx, kx, torch, sizes=(32, 64, 96, 128, 192, 256, 384, 512),
                          check_max_n=256, iters=20):
    """The paper's runtime benchmark (Sec. 5, Fig. run_time): one full-grid
    evaluation of the elastic self-collision operator for the two-bump f of
    eq. (benchmark_two_bump) with m = 1, a = 1, q in [1e-3, 1e2], N_mu = 18,
    Bose-Einstein factors and no projection, as a function of N; device time
    of the whole evaluation (prepare f, contraction, row combine) replayed as a
    CUDA graph, warm caches, on the plain FP64 and the FP32 path.  Returns the
    line and the outputs at N <= check_max_n (compared with the FP64 oracle in
    the CPU-baseline leg)."""
    rows, check = [], []
    for n in sizes:
        q = ki.log_grid(n, 1e-3, 1e2)
        f = ki.paper_two_bump(q)
        fd = torch.as_tensor(f[None], device="cuda")
        row = {"n": n}
        outs = {}
        for name, prec in (("fp64", kx.FP64), ("fp32", kx.FP32)):
            k = ctx.build_kernel(q, precision=prec, stats=1)
            ms, C = ctx.time_collision(k, fd, 1.0, project=False, iters=iters)
            row[name + "_us_per_eval"] = 1e3 * ms
            outs[name] = C.cpu().numpy()[0]
            k.release()
        row["speedup_fp32_vs_fp64"] = row["fp64_us_per_eval"] / row["fp32_us_per_eval"]
        rows.append(row)
        if n <= check_max_n:
            check.append({"n": n, "q": q, "f": f, "C": outs, "row": row})
    line = {"workload": "Fig. run_time of the paper: eq. (benchmark_two_bump), m=1, a=1, "
                        "q in [1e-3,1e2], N_mu=18, Bose-Einstein factors, no projection; one "
                        "full-grid evaluation (graph replay, warm caches)",
            "rows": rows}
    return line, check


def oracle_errors(batched_check, runtime_check):
    """CPU-baseline leg: the FP64 oracle on the samples the GPU lines kept;
    max relative error (max-norm over the grid) of each path against it."""
    import oracle
    out = {}
    if batched_check is not None:
        q, f, sig = batched_check["q"], batched_check["f"], batched_check["sigma"]
        W = oracle.kernel_tensor(q)
        g = oracle.grid(q)
        err = {name: 0.0 for name in batched_check["C"]}
        for b in range(f.shape[0]):
            M2 = oracle.M2_from_sigma(1.0, sig[b])
            Co, _ = oracle.project(g["E"], g["h"], f[b], oracle.collision_tensor(q, W, f[b]) * M2)
            Cq, _ = oracle.project(g["E"], g["h"], f[b], oracle.collision_tensor_stats(q, W, f[b], 1) * M2)
            for name, C in batched_check["C"].items():
                ref = Cq if name.endswith("bose_einstein") else Co
                err[name] = max(err[name], float(np.max(np.abs(C[b] - ref)) / np.max(np.abs(ref))))
        out["batched"] = err
    for item in runtime_check or []:
        q, f = item["q"], item["f"]
        Co = oracle.collision_tensor_stats(q, oracle.kernel_tensor(q), f, 1) * oracle.M2_from_sigma(1.0, 1.0)
        for name, C in item["C"].items():
            item["row"][name + "_max_rel_err_vs_oracle"] = float(np.max(np.abs(C - Co)) / np.max(np.abs(Co)))
    return out


def measure_config1(ctx, kx, torch, reps=5):
    """Single instance, N = 32 (q in [1e-3, 10]), sigma = 1: 100 fixed Heun
    steps of h = 0.02 per solve (2 evaluations a step), on the plain FP64 and
    the FP32 path; steps/s from CUDA events around `reps` solves, and the
    contraction alone (warm L2, the kernel is 0.3 MB)."""
    c = ki.config1()
    q, f0 = c["q"], c["f0"]
    out = {"workload": "N=32, q in [1e-3,10], sigma=1, 100 fixed Heun steps (h=0.02) from the "
                       "seeded bimodal f"}
    for name, prec in (("fp64", kx.FP64), ("fp32", kx.FP32)):
        k = ctx.build_kernel(q, precision=prec)
        fd = torch.as_tensor(np.tile(f0, (1, 1)), device="cuda")
        kw = dict(t_end=c["n_steps"] * c["h"], h0=c["h"], fixed_step=1)
        ctx.solve(k, fd.clone(), c["sigma"], **kw)              # warm (graph capture, tuning)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        steps = 0
        for _ in range(reps):
            f = fd.clone()
            res = ctx.solve(k, f, c["sigma"], **kw)
            steps += res[0]["steps"]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        us_c = 1e3 * ctx.time_contraction(k, fd, iters=50, flush_bytes=0)
        k.release()
        out[name] = {"steps_per_s": steps / (ms * 1e-3), "us_per_step": 1e3 * ms / steps,
                     "us_per_eval": 1e3 * ms / (2 * steps), "contraction_us": us_c}
    out["speedup_fp32_vs_fp64_steps"] = out["fp32"]["steps_per_s"] / out["fp64"]["steps_per_s"]
    return out


def measure_grouped(ctx, kx, c, par, t_end, forms=(0, 16)):
    """The uneven batch as one sequence of grouped launches (kx_solve_grouped:
    per Heun stage one gain-GEMM launch, one loss launch (Chebyshev GEMM, or the
    grids' exact loss kernels side by side) and one stage launch over all five
    grids, captured in a graph of attempts), exact loss and Chebyshev K = 16."""
    import torch
    sizes = (64, 96, 128, 192, 256)
    grouped = {}
    for lt in forms:
        ks = [ctx.build_kernel(c["grids"][n], precision=kx.SPLIT_TF32, loss_terms=lt) for n in sizes]
        idx = [np.nonzero(c["ns"] == n)[0] for n in sizes]
        fs = [torch.as_tensor(np.stack([c["f"][i] for i in ii]), device="cuda") for ii in idx]
        sg = [c["sigma"][ii] for ii in idx]
        gp = dict(par, t_end=t_end, h0=1e-3)
        ctx.solve_grouped(ks, [f.clone() for f in fs], sg, **dict(gp, t_end=1e-3))   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.solve_grouped(ks, fs, sg, **gp)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        done = sum(1 for r in res for x in r if x["status"] == 0)
        evals = sum(x["evals"] for r in res for x in r)
        grouped["cheb16" if lt else "exact_loss"] = {
            "instances": len(c["ns"]), "completed": done, "seconds": dt, "solves_per_s": done / dt,
            "evals_per_s": evals / dt, "evals": evals}
        for k in ks:
            k.release()
    return grouped


def measure_uneven(ctx, kx, t_end=5.0, fp64_per_size=4):
    """Uneven batch: 1024 instances with N uniform over {64, 96, 128, 192, 256},
    sigma log-uniform over [1e-3, 1], 5 shared kernel tensors, all admitted at once
    into the solve server (one group and one captured graph of attempts per
    kernel, groups on concurrent streams), split-TF32 tensor-core path; each
    instance integrated to t = t_end.  The plain FP64 path is timed on a sample of
    the same instances through the same server."""
    c = ki.config4()
    par = dict(rtol=1e-6, atol=1e-12, l1_tol=0.0, check_every=10, max_attempts=1_000_000)
    out = {}
    for name, prec, idx in (("split_tf32", kx.SPLIT_TF32, range(len(c["ns"]))),
                            ("fp64", kx.FP64, None)):
        if idx is None:   # a few instances of each size
            idx = [i for n in (64, 96, 128, 192, 256)
                   for i in np.nonzero(c["ns"] == n)[0][:fp64_per_size]]
        srv = kx.Server(ctx, budget_bytes=64 << 30, slots_per_group=256, attempts_per_tick=8,
                        precision=prec, **par)
        # build the five kernels first (cold builds are reported separately)
        tb = time.perf_counter()
        warm = [srv.submit(c["grids"][n], c["f"][int(np.nonzero(c["ns"] == n)[0][0])], 1.0,
                           t_end=1e-9, h0=1e-3) for n in (64, 96, 128, 192, 256)]
        for t, n in zip(warm, (64, 96, 128, 192, 256)):
            srv.poll(t, n, timeout=600.0)
        t_build = time.perf_counter() - tb
        ev0 = srv.stats()["evals"]
        t0 = time.perf_counter()
        tickets = [(srv.submit(c["grids"][int(c["ns"][i])], c["f"][i], float(c["sigma"][i]),
                               t_end=t_end, h0=1e-3), int(c["ns"][i])) for i in idx]
        ok = 0
        for t, n in tickets:
            rc, _, _ = srv.poll(t, n, timeout=1800.0)
            ok += rc == kx.OK
        dt = time.perf_counter() - t0
        st = srv.stats()
        srv.stop()
        evals = st["evals"] - ev0
        out[name] = {"instances": len(tickets), "completed": ok, "seconds": dt,
                     "solves_per_s": ok / dt, "evals_per_s": evals / dt, "evals": evals,
                     "kernel_build_s": t_build}
    grouped = measure_grouped(ctx, kx, c, par, t_end)
    return {"workload": "1024 instances, N uniform over {64,96,128,192,256}, sigma logU[1e-3,1], "
                        f"no sources, each integrated to t={t_end}; all admitted at once",
            "split_tf32": out["split_tf32"], "fp64_path_sample": out["fp64"],
            "speedup_vs_fp64_evals": out["split_tf32"]["evals_per_s"] / out["fp64"]["evals_per_s"],
            "grouped_launch": grouped,
            "grouped_speedup_vs_fp64_evals": {k2: v2["evals_per_s"] / out["fp64"]["evals_per_s"]
                                              for k2, v2 in grouped.items()},
            "note": "split_tf32: the solve server (one group and captured graph per grid, groups "
                    "on concurrent streams); grouped_launch: kx_solve_grouped, one launch per "
                    "phase over all grids; fp64_path_sample: the server on the plain FP64 path"}


def serve_stream(kx, ctx, reqs, precision, budget=96 << 30, slots=2, phases=("run",)):
    """Submit `reqs` at their arrival times to one server; one result dict per phase
    (the same stream again in each phase, kernels cached after the first)."""
    par = dict(rtol=1e-6, atol=1e-12, l1_tol=1e-3, check_every=10, max_attempts=2_000_000)
    srv = kx.Server(ctx, budget_bytes=budget, slots_per_group=slots, attempts_per_tick=8,
                    precision=precision, **par)
    res = {}
    for phase in phases:
        srv.reset_latency()   # this phase's latency quantiles only
        s0 = srv.stats()
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = r["arrival"] - reqs[0]["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append((srv.submit(r["q"], r["f0"], r["sigma"], sources=r["sources"],
                                       t_end=1e5, h0=1e-3), r["n"]))
        lat, ok, conv = [], 0, 0
        for t, n in tickets:
            rc, _, rr = srv.poll(t, n, timeout=3600.0)
            if rc == kx.OK:
                ok += 1
                conv += int(rr["converged"])
                lat.append(rr["latency_s"])
        dt = time.perf_counter() - t0
        s1 = srv.stats()
        res[phase] = {"requests": len(reqs), "completed": ok, "converged": conv,
                      "failed": len(reqs) - ok, "seconds": dt, "solves_per_s": ok / dt,
                      "converged_solves_per_s": conv / dt,
                      "evals_per_s": (s1["evals"] - s0["evals"]) / dt,
                      "p50_latency_s": float(np.percentile(lat, 50)) if lat else None,
                      "p99_latency_s": float(np.percentile(lat, 99)) if lat else None,
                      # the server's split of this phase's latencies into the wait
                      # for a slot (submit to admission) and the service (admission
                      # to result)
                      "p50_queue_wait_s": s1["p50_wait_s"], "p99_queue_wait_s": s1["p99_wait_s"],
                      "p50_service_s": s1["p50_service_s"], "p99_service_s": s1["p99_service_s"],
                      "ticks_shared": s1["ticks_shared"] - s0["ticks_shared"],
                      "ticks_whole": s1["ticks_whole"] - s0["ticks_whole"],
                      # the completed solves' table bytes (one pass per evaluation)
                      # per second: an upper bound of the algorithmic HBM read rate
                      "stream_gbs": (s1["stream_bytes"] - s0["stream_bytes"]) / dt / 1e9,
                      "kernels_built": s1["kernels_built"] - s0["kernels_built"],
                      "kernel_cache_hits": s1["kernel_cache_hits"] - s0["kernel_cache_hits"]}
    srv.stop()
    return res


def measure_serving(ctx, kx, requests=200, fp64_requests=16):
    """Serving: a seeded Poisson stream (mean 200 req/s) of full solves with
    N ~ U{64..384}, sigma ~ logU[1e-2, 10], random initial and source bumps,
    submitted at their arrival times.  FP32 path: kernel tensors built on demand
    (cold), then the same stream with every kernel cached (warm).  The plain FP64
    path and the FP32 path also serve the stream's first `fp64_requests` requests
    (same inputs, cold) for the speedup.  The configured stream has 2000
    requests; `requests` takes its first ones (the default keeps the bench within
    minutes; --requests 2000 serves all of them)."""
    reqs = ki.config5()[:requests]
    out = serve_stream(kx, ctx, reqs, kx.FP32, phases=("cold", "warm"))
    sub = reqs[:fp64_requests]
    a = serve_stream(kx, ctx, sub, kx.FP32)["run"]
    b = serve_stream(kx, ctx, sub, kx.FP64)["run"]
    out["same_inputs_fp32"] = a
    out["same_inputs_fp64_path"] = b
    hbm, src = peaks()
    if "warm" in out:
        w = out["warm"]["stream_gbs"]
        out["roofline"] = {"bound": "hbm", "achieved": w, "peak": hbm, "unit": "GB/s", "frac": w / hbm,
                           "phase": "warm", "peak_source": src,
                           "note": "the completed solves' evaluations x their kernel's streamed table "
                                   "bytes per second: an upper bound of the algorithmic reads (the two "
                                   "slots of a group share a pass; tables of the smaller grids can stay "
                                   "in the 126 MB L2), so the fraction is an upper bound too"}
    out["speedup_vs_fp64_solves_per_s"] = (a["solves_per_s"] / b["solves_per_s"]
                                           if b["solves_per_s"] > 0 else None)
    out["speedup_vs_fp64_converged_solves_per_s"] = (a["converged_solves_per_s"] / b["converged_solves_per_s"]
                                                     if b["converged_solves_per_s"] > 0 else None)
    out["workload"] = (f"first {requests} of the 2000-request Poisson stream (200 req/s), "
                       "N ~ U{64..384}, sigma logU[1e-2,10], two random source bumps each, full "
                       "solves to L1<=1e-3 after the sources are off (t_end = 1e5); FP32 path, 2 "
                       f"slots per kernel group; FP32 vs FP64 path on the first {fp64_requests} "
                       "requests")
    if requests < 2000:
        out["prefix_reason"] = ("the full 2000-request stream takes several minutes per phase; "
                                "bench.py --only serving --requests 2000 serves all of it")
    return out


def aggregate_ranks(dist, total_ms, evals, solves, device):
    """Whole-job figures of N independent replicas (one per rank, weak scaling):
    the slowest rank's timed milliseconds and the work summed over ranks.  No
    data-path collective: the ranks exchange only these three numbers."""
    if dist is None:
        return total_ms, evals, solves
    import torch
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    cnt = torch.tensor([evals, solves], device=device, dtype=torch.float64)
    dist.all_reduce(cnt)
    return float(t.item()), int(cnt[0].item()), int(cnt[1].item())


def config_desc(c, B):
    return {"workload": "single instance N=128 full integration: kernel build + adaptive Heun "
                        "solve with two freeze-in sources for sigma in {0.1,1,10,100} "
                        "(batch of 4 sharing one kernel) to L1<=1e-3 vs MB",
            "n": int(c["q"].size), "batch": B, "q_range": [1e-3, 10.0], "mass": 1.0,
            "n_mu": 18, "path": "FP32 streaming contraction, FP64 projection/stepper",
            "l2": "flushed between timed steps (512 MB write)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default="", choices=["", "contraction", "step", "uneven", "serving", "batched",
                                                   "grouped"],
                    help="contraction: time the contraction kernel alone; step: run the "
                         "workload's steps only (no baselines), for profiling")
    ap.add_argument("--n", type=int, default=384)
    ap.add_argument("--qmax", type=float, default=1e2,
                    help="--only contraction: the grid's largest q/m (the N=128 workload uses 10)")
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "split"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--pdl", action="store_true",
                    help="--rotate: launch with programmatic dependent launch")
    ap.add_argument("--rotate", type=int, default=0,
                    help="--only contraction: time R kernels of the grid back to back in rotation")
    ap.add_argument("--variant", type=int, default=-1,
                    help="FP32: pin the streaming variant (0..4) instead of tuning it")
    ap.add_argument("--requests", type=int, default=200,
                    help="serving: the first R requests of the 2000-request stream")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the uneven-batch and serving measurements")
    ap.add_argument("--no-split-tuning", action="store_true",
                    help="split path: the default launch choices, not timed ones (for profiling)")
    ap.add_argument("--paper-runtime", action="store_true",
                    help="also re-time the paper's own runtime figure (one evaluation vs N, "
                         "Bose-Einstein factors; context only)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.only == "contraction":
        return run_contraction_only(args)
    if args.only in ("uneven", "serving", "batched", "grouped"):
        import torch
        import paper_2607_00755_b300 as kx
        ctx = kx.Context(0)
        if args.no_split_tuning:
            ctx.set_split_tuning(False)
        if args.only == "batched":
            flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
            r = measure_batched(ctx, kx, torch, flush)[0]
        elif args.only == "grouped":
            r = measure_grouped(ctx, kx, ki.config4(), dict(rtol=1e-6, atol=1e-12, l1_tol=0.0, check_every=10,
                                                            max_attempts=1_000_000), 5.0)
        else:
            r = measure_uneven(ctx, kx) if args.only == "uneven" else measure_serving(
                ctx, kx, requests=args.requests)
        print(json.dumps(r), flush=True)
        ctx.close()
        return 0

    import torch
    import paper_2607_00755_b300 as kx
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = kx.Context(local)
    stream = torch.cuda.current_stream()
    c, B, f0, par = workload()
    q, sig, src = c["q"], c["sigmas"], c["sources"]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def one_step(precision):
        k = ctx.build_kernel(q, precision=precision)
        fd = torch.as_tensor(f0, device="cuda")
        res = ctx.solve(k, fd, sig, sources=src, **par)
        k.release()
        return res

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.variant >= 0:   # (profiling: a serialising profiler would tune differently)
        ctx.set_stream_variant(len(q), B, args.variant)
    for _ in range(args.warmup):
        one_step(kx.FP32)
    if args.only == "step":
        for _ in range(args.steps):
            one_step(kx.FP32)
        torch.cuda.synchronize()
        ctx.close()
        return 0
    uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    barrier()
    clocks = ClockSampler(uuid)
    launches0 = ctx.launch_count()
    total_ms, evals, solves, results = 0.0, 0, 0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()                      # cold L2 before each step (not timed)
        e0.record(stream)
        res = one_step(kx.FP32)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        evals += sum(r["evals"] for r in res)
        solves += len(res)
        results += res
    barrier()
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    t_local = total_ms
    total_ms, evals, solves = aggregate_ranks(dist, total_ms, evals, solves, "cuda")
    value = evals / (total_ms / 1e3)
    solves_per_s = solves / (total_ms / 1e3)
    bad = [r for r in results if r["status"] != 0 or not r["converged"]]

    # ---- end to end through the public API with host buffers ------------------
    e2e_t, e2e_evals = 0.0, 0
    h2d = q.nbytes + f0.nbytes + src["shape"].nbytes * 1
    d2h = f0.nbytes
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = ctx.build_kernel(q, precision=kx.FP32)
        fh, res = ctx.solve_host(k, f0, sig, sources=src, **par)
        k.release()
        torch.cuda.synchronize()
        e2e_t += time.perf_counter() - t0
        e2e_evals += sum(r["evals"] for r in res)

    # ---- plain FP64 path on the same inputs ------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        one_step(kx.FP64)
        t64, ev64 = 0.0, 0
        for _ in range(args.fp64_steps):
            flush.zero_()
            e0.record(stream)
            res = one_step(kx.FP64)
            e1.record(stream)
            e1.synchronize()
            t64 += e0.elapsed_time(e1)
            ev64 += sum(r["evals"] for r in res)
        fp64 = {"value": ev64 / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / args.fp64_steps,
                "solves_per_s": B * args.fp64_steps / (t64 / 1e3)}

    # ---- rooflines of the step's two kernels, timed live --------------------
    # The solve runs the four instances as concurrent chains (one instance per
    # launch).  kx_profile_attempts runs real Heun attempts of one chain (the
    # longest, sigma = 0.1) with CUDA events between its contraction and stage
    # kernels (plain stream order: each time includes the kernel's launch and
    # its wait on the predecessor, and no other chain runs beside it); the FP64
    # and ex2 peaks come from the library's throughput kernels in this run
    # (FP64: FMA = 2 flops)
    hbm, src_peak = peaks()
    fp64_peak, ex2_peak = ctx.measure_peaks()
    kk = ctx.build_kernel(q, precision=kx.FP32)
    Bp = 1
    fprof = torch.as_tensor(f0[:Bp], device="cuda")
    prof = ctx.profile_attempts(kk, fprof, sig[:Bp], sources=src, attempts=400, **par)
    info = kk.info()
    alg_bytes = info["stream_bytes"]
    kname = stream_kernel_name(ctx, 128, Bp)
    us_k = 0.5 * (prof["contraction_1_us"] + prof["contraction_2_us"])
    us_s = 0.5 * (prof["stage_1_us"] + prof["stage_2_us"])
    ms_cold = ctx.time_contraction(kk, torch.as_tensor(f0, device="cuda"), iters=30,
                                   flush_bytes=L2_FLUSH_BYTES)
    kk.release()
    n = q.size
    # contraction: the method's one exponential per kept element and instance (the
    # interpolated f_t); the kernel evaluates two ex2 per element (the
    # 2^a (1 - 2^d) form)
    elem = info["nonzero_elements"] * Bp
    tr_k, tr_k_note = traffic_for("stream_n128_b1", kname.split(" ")[0], alg_bytes)
    roof_k = {"bound": "alu", "pipe": "MUFU (ex2)", "achieved": elem / (us_k * 1e-6) / 1e12,
              "peak": ex2_peak / 1e12, "unit": "Tex2/s", "frac": elem / (us_k * 1e-6) / ex2_peak,
              "traffic": tr_k, "traffic_note": tr_k_note,
              "kernel": f"N=128, one chain (1 instance): {kname}", "elements_per_launch": elem,
              "avg_launch_us": us_k, "avg_launch_ms_isolated_cold_l2": ms_cold,
              "algorithmic_bytes_per_launch": alg_bytes,
              "l2_resident": "the tables (%.1f MB) stay in the 126 MB L2 during the solve" % (alg_bytes / 1e6),
              "issued_frac": 2 * elem / (us_k * 1e-6) / ex2_peak,
              "note": "latency and issue bound at this size: each warp streams 2-3 units of its "
                      "bins after loading the instance tables written by the previous stage"}
    flop_s = Bp * n * 0.5 * (STAGE_FLOP_PER_POINT[1] + STAGE_FLOP_PER_POINT[2])
    tr_s, tr_s_note = traffic_for("stage_n128_b1", "k_stage<1,0>")
    roof_s = {"bound": "alu", "pipe": "FP64", "achieved": flop_s / (us_s * 1e-6) / 1e9,
              "peak": fp64_peak / 1e9, "unit": "GFLOP/s", "frac": flop_s / (us_s * 1e-6) / fp64_peak,
              "traffic": tr_s, "traffic_note": tr_s_note,
              "kernel": "k_stage<1,0>: one block per instance (one chain: 1 block), row combine, "
                        "projection, Heun stage, MB check, next tables",
              "flop_per_launch": flop_s, "avg_launch_us": us_s,
              "frac_of_the_sms_it_occupies": flop_s / (us_s * 1e-6) / (fp64_peak * Bp / 148.0),
              "note": "latency bound: a dependent chain of FP64 operations and block reductions "
                      "per instance on one SM each"}
    dominant = "stage" if us_s >= us_k else "contraction"
    roof = dict(roof_s if dominant == "stage" else roof_k)
    roof["dominant"] = (f"{dominant}: {max(us_s, us_k):.2f} us of the {us_s + us_k:.2f} us of the "
                        "two kernels per Heun stage of one chain (kx_profile_attempts, 400 attempts)")
    roof["peak_source"] = "measured in this run (the library's DFMA / ex2 throughput kernels)"
    roof_other = roof_k if dominant == "stage" else roof_s
    roof_other["peak_source"] = roof["peak_source"]
    # streaming single-instance rooflines at N=384 and N=512 (tables 172 MB
    # and 406 MB, both > L2): several kernels of the same grid whose
    # contractions run back to back in rotation, so that each launch streams
    # its tables from HBM (about 1 GB read between two launches of one
    # kernel); the isolated launch after an L2 flush beside it
    def streaming_roofline(n, rotate):
        qn = ki.log_grid(n, 1e-3, 1e2)
        ks = [ctx.build_kernel(qn, precision=kx.FP32) for _ in range(rotate)]
        fn = torch.as_tensor(ki.batch_bimodal(np.random.default_rng(7), qn, 1), device="cuda")
        ms_rot = ctx.time_contractions(ks, fn, iters=10)
        ms_pdl = ctx.time_contractions(ks, fn, iters=10, pdl=True)
        ms_iso = ctx.time_contraction(ks[0], fn, iters=20, flush_bytes=L2_FLUSH_BYTES)
        nb = ks[0].info()["stream_bytes"]
        for kr in ks:
            kr.release()
        gbs = nb / (ms_pdl * 1e-3) / 1e9
        kn = stream_kernel_name(ctx, n, 1)
        tr, tr_note = traffic_for(f"stream_n{n}", kn.split(" ")[0], nb)
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": tr, "traffic_note": tr_note, "peak_source": src_peak,
                "kernel": f"N={n}, single instance: {kn}",
                "algorithmic_bytes_per_launch": nb, "avg_launch_ms": ms_pdl,
                "timing": f"{rotate} kernels of the grid ({rotate} x {nb / 1e6:.0f} MB tables) in "
                          f"rotation, {10 * rotate} launches back to back between CUDA events, "
                          "launched as inside the solve's graphs (programmatic dependent launch: "
                          "a launch's first table loads overlap its predecessor's tail)",
                "avg_launch_ms_stream_order": ms_rot,
                "frac_stream_order": nb / (ms_rot * 1e-3) / 1e9 / hbm,
                "avg_launch_ms_isolated_cold_l2": ms_iso,
                "frac_isolated_cold_l2": nb / (ms_iso * 1e-3) / 1e9 / hbm,
                "evals_per_s": 1e3 / ms_pdl}

    roof384 = streaming_roofline(384, 6)
    roof512 = streaming_roofline(512, 3)

    config1 = measure_config1(ctx, kx, torch) if rank == 0 else None
    batched, batched_check = measure_batched(ctx, kx, torch, flush) if rank == 0 else (None, None)
    runtime, runtime_check = (measure_paper_runtime(ctx, kx, torch)
                              if rank == 0 and args.paper_runtime else (None, None))
    uneven = measure_uneven(ctx, kx) if rank == 0 and not args.no_serving else None
    serving = (measure_serving(ctx, kx, requests=args.requests)
               if rank == 0 and not args.no_serving else None)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        e, t, cores = oracle_sample(c, B, 12.0)
        # the same sample on one thread, and the host's CPU model
        import oracle
        oracle.set_threads(1)
        e1, t1, _ = oracle_sample(c, B, 4.0)
        oracle.set_threads(cores)
        cpu = {"value": e / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{e} RHS evaluations (tensor-form C + projection + sources) of the "
                         f"N=128 workload's first Heun attempts in {t:.1f} s",
               "single_thread_value": e1 / t1, "cpu_model": cpu_model()}
        errs = oracle_errors(batched_check, runtime_check)
        if batched is not None:
            batched["max_rel_err_vs_oracle"] = errs.get("batched")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_desc(c, B),
                "solves_per_s": solves_per_s,
                "fp64_path": fp64,
                "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
                "failed_solves": len(bad),
                "per_instance": [{"sigma": float(sig[b]), "steps": int(results[b]["steps"]),
                                  "rejects": int(results[b]["rejects"]),
                                  "evals": int(results[b]["evals"]), "t": results[b]["t"],
                                  "l1_to_mb": results[b]["l1_to_mb"]}
                                 for b in range(min(B, len(results)))],
                "roofline": roof, "roofline_other_kernel": roof_other,
                "roofline_streaming_n384": roof384,
                "roofline_streaming_n512": roof512,
                "fixed_steps_n32": config1,
                "batched_n192_b512": batched,
                "paper_runtime_bose_einstein": runtime,
                "uneven_batch": uneven,
                "serving": serving,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_evals / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    del t_local
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

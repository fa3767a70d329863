"""Benchmark: milliseconds to a normwise relative backward error <= 1e-15 for a dense n = 16384
system with recycled mixed-precision GMRES-IR (FP16 tensor-core LU with diagonal scaling -- the
paper's half precision --, FP64 working precision and residual, GCRO-DR(50, 10)), on synthetic
randsvd matrices (geometric singular values, kappa_2 = 1e2). The same system with a BF16 LU, with
k = 0 (GMRES-IR), a prolate matrix where recycling pays, and an FP64 LU solve are reported beside
it as comparators.

One step = the whole hot path on one system: gir_factor (scaling, u_f LU, diagonal-block
inverses) + gir_solve (x0, refinement steps with FP64 residuals, GCRO-DR corrections) with
A and b already resident in HBM. `e2e` times the same call sequence through the C ABI with
the inputs in pinned host memory and the host<->device copies inside the timed region.
The CPU oracle is timed on a bounded sample (a smaller system of the same family) and scaled
by n^3 to the benchmark size.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to 1e-15 rel. backward error, n=16384: recycled GMRES-IR vs FP64 LU"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gir_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(n_s=3072, kappa=1e2, uf="bf16"):
    """The CPU oracle (as it stands) on one system of the benchmark family at size n_s."""
    import numpy as np
    from oracle.ir import Params as OP, solve as osolve
    from synth import randsvd, normal_vector
    A = randsvd(n_s, kappa, seed=0)
    b = A @ normal_vector(n_s, 2)
    t = time.perf_counter()
    x, info, _, _ = osolve(A, b, OP(uf=uf, u="fp64", ur="fp64", ua="u", m=50, k=10, tau=1e-8, imax=10,
                                    target=1e-15, lu_w=32))
    dt = time.perf_counter() - t
    return dt, info


def oracle_projection(n, n_s, kappa, uf):
    """The oracle at n_s / 2 and n_s; the time at n from the exponent fitted to the two points
    (the LU is O(n^3), the refinement O(n^2) per iteration, so the exponent lies between)."""
    import math
    t1, i1 = oracle_sample(n_s // 2, kappa, uf)
    t2, i2 = oracle_sample(n_s, kappa, uf)
    expo = math.log(t2 / t1) / math.log(2.0)
    return t2 * (n / n_s) ** expo, t1, t2, expo, i1, i2


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_json(n, n_s, kappa, uf):
    proj, t1, t2, expo, i1, i2 = oracle_projection(n, n_s, kappa, uf)
    return {"value": proj * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle RGMRES-IR (numpy FP64, u_f by rounding) on randsvd kappa_2={kappa:g}, {uf}, "
                      f"GCRO-DR(50,10) at n={n_s // 2} ({t1:.2f} s, {i1.paper_format()}) and n={n_s} "
                      f"({t2:.2f} s, {i2.paper_format()}); time at n={n} projected with the fitted exponent "
                      f"{expo:.2f}; host CPU {cpu_model()}"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_s = args.sample_n
    vals = []
    for _ in range(args.warmup):
        oracle_sample(max(256, n_s // 4), args.kappa, args.uf)
    expos = []
    for _ in range(args.steps):
        proj, t1, t2, expo, _, _ = oracle_projection(args.n, n_s, args.kappa, args.uf)
        vals.append(proj * 1e3)
        expos.append(expo)
    v = statistics.median(vals)
    cb = {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"oracle RGMRES-IR on randsvd at n={n_s // 2} and n={n_s} per step, projected to n={args.n} "
                    f"with the fitted exponent (median {statistics.median(expos):.2f}); host CPU {cpu_model()}"}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_json(args, world), "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def config_json(args, world):
    return {"workload": f"randsvd dense n={args.n}, kappa_2={args.kappa:g}, b=A x*, x*~N(0,1); "
                        f"u_f={args.uf} LU (tcgen05), u=fp64, u_r=fp64, GCRO-DR(m={args.m},k={args.k}), tau=1e-8, "
                        f"target berr 1e-15",
            "n": args.n, "kappa_2": args.kappa, "uf": args.uf, "u": "fp64", "ur": "fp64", "m": args.m, "k": args.k,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (A is 8n^2 bytes = 2.15 GB at n=16384)"}


# Algorithmic work of the traced kernels: per-unit figures times the units of all launches of
# the step (the per-launch figure is the total over the step divided by the launch count).
FP32_ALU_TFLOPS_DERIVED = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
# the phases timed inside the timed region (the dominant kernel and the next ones)
ROOFLINE_PHASES = ["lu panel", "trsv", "gemv", "lu outer gemm"]


def phase_work(phase, args, calls):
    """(total algorithmic units over all launches of the step, unit, bound) or None."""
    n, nb, w = args.n, 256, 32
    steps = max(1, args.steps)
    if phase == "lu panel":
        # read the FP32 panel, write it back and its u_f copy: 10 bytes per panel entry
        tot = sum(10.0 * (n - c0) * min(w, n - c0) for c0 in range(0, n, w))
        return steps * tot, "GB/s", "hbm"
    if phase == "trsv":
        # one triangle of the 16-bit factors (n^2 / 2 entries) plus the right-hand side and result
        return calls * (1.0 * n * n + 24.0 * n), "GB/s", "hbm"
    if phase == "gemv":
        return calls * (8.0 * n * n + 16.0 * n), "GB/s", "hbm"
    if phase == "residual":
        return calls * (8.0 * n * n + 24.0 * n), "GB/s", "hbm"
    if phase == "lu outer gemm":
        tot = sum(2.0 * (n - c) * (n - c) * nb for c in range(nb, n, nb))
        return steps * tot, "TFLOP/s", "tensor"
    if phase == "lu outer trsm":
        # FP32 substitution of the U12 band: nb^2 fused multiply-adds per trailing column
        tot = sum(2.0 * nb * nb / 2 * (n - c) for c in range(nb, n, nb))
        return steps * tot, "TFLOP/s", "alu"
    return None


def read_traffic(kernel_phase):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel's source
    changed since the capture (the summary records a hash of the file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0].replace("_", " ") == kernel_phase:
            src = os.path.join(ROOT, "paper_2201_09827_gb300", "csrc", parts[2])
            try:
                h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            except OSError:
                return None
            return float(parts[1]) if h == parts[3] else None
    return None


def roofline_for(phase, total_ms, calls, args, peaks, peak_kind):
    work = phase_work(phase, args, calls)
    if work is None:
        return None
    tot, unit, bound = work
    per = tot / max(calls, 1)
    avg_s = (total_ms / calls) * 1e-3
    if unit == "GB/s":
        achieved, pk, pk_src = per / avg_s / 1e9, peaks["hbm_gbs"], f"hbm_gbs of {peak_kind}"
    elif bound == "tensor":
        achieved, pk, pk_src = per / avg_s / 1e12, peaks["bf16_tflops"], f"bf16_tflops (burst) of {peak_kind}"
    else:
        achieved, pk, pk_src = per / avg_s / 1e12, FP32_ALU_TFLOPS_DERIVED, "derived FP32 FMA peak"
    return {"kernel": phase, "bound": bound, "achieved": achieved, "peak": pk, "unit": unit, "frac": achieved / pk,
            "traffic": read_traffic(phase), "peak_source": pk_src, "per_launch": per, "launches": calls,
            "avg_ms": total_ms / calls}


def sweep_line(args, world, workload, extra_cfg, ms, times, result, roof=None, cpu=None, e2e=None, clocks=None,
               launches=None, metric=METRIC):
    """One JSON line of the measurement matrix, with the keys of the headline line."""
    cfg = {"workload": workload, **extra_cfg,
           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
           "l2": "inputs larger than L2 where the matrix exceeds 129 MB; smaller ones run from L2"}
    return {"metric": metric, "value": ms, "unit": "ms", "n_gpus": world, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "e2e": e2e,
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "result": {**result, "times_ms": times}, "sweep": True}


def run_sweep(args, rank, world, local):
    """The measurement matrix: every point runs W untimed and K timed steps (factor + solve with
    the inputs resident in HBM, CUDA events on the launching stream), median reported."""
    import torch
    import numpy as np
    import paper_2201_09827_gb300 as gir
    from synth import randsvd_torch, prolate, convdiff, rhs_uniform, normal_vector, batch_specs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    out = []

    def emit(line):
        if rank == 0:
            print(json.dumps(line), flush=True)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts, res = [], None
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), ts, res

    def solve_step(A, b, prm):
        def fn():
            F = gir.Factorization(A, prm)
            x, info = F.solve(A, b)
            F.close()
            return x, info
        return fn

    def berr_dd(A, x, b):
        r = gir.residual(A, x, b, "dd")
        return (r.abs().max() / (A.abs().sum(1).max() * x.abs().max() + b.abs().max())).item()

    n = args.n
    parts = set(args.only.split(",")) if args.only else {"randsvd", "prolate", "convdiff", "batch", "oracle"}
    # (batch-small, the 24-system counter-capture workload, and adjoint, the transposed solves against
    # the forward ones, run only when named)
    # ---- headline matrix: kappa_2 x u_f, RGMRES-IR(50, 10) and the GMRES-IR(50) comparator
    for kappa in ((1e2, 1e4, 1e6, 1e8) if "randsvd" in parts else ()):
        A = randsvd_torch(n, kappa, seed=0, device=f"cuda:{local}")
        g = torch.Generator(device=dev)
        g.manual_seed(2)
        xstar = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        b = A @ xstar
        for uf in ("fp16", "bf16", "e4m3"):
            # GCRO-DR(50, 10) against GMRES(50), and GCRO-DR(100, its_1 - 1) (the recycle dimension of
            # Section 5, GIR_FLAG_ADAPTIVE_K) against GMRES(100); Arnoldi steps capped at 4 m per step
            for m, k, adaptive in ((args.m, args.k, False), (args.m, 0, False), (100, 0, True), (100, 0, False)):
                flags = gir.GIR_FLAG_ADAPTIVE_K if adaptive else 0
                prm = gir.Params(uf=uf, u="fp64", ur="fp64", m=m, k=k, tau=1e-8, imax=10, target_berr=1e-15,
                                 carry_mode=1, max_its=4 * m, flags=flags)
                first = solve_step(A, b, prm)()
                steps = args.steps if first[1].status == 0 else 1     # a stagnating run is timed once
                ms, ts, (x, info) = timed(solve_step(A, b, prm), steps, 0)
                ferr = ((x - xstar).abs().max() / xstar.abs().max()).item()
                name = ("RGMRES-IR" if (k or adaptive) else "GMRES-IR") + f"(m={m}, k={'its_1-1' if adaptive else k})"
                emit(sweep_line(args, world, f"randsvd dense n={n}, kappa_2={kappa:g}, b=A x*; u_f={uf}, u=u_r=fp64, "
                                             f"{name}, tau=1e-8, target berr 1e-15, <= {4 * m} Arnoldi steps per "
                                             f"refinement step, i_max=10",
                                {"n": n, "kappa_2": kappa, "uf": uf, "u": "fp64", "ur": "fp64", "m": m,
                                 "k": "its_1-1" if adaptive else k, "max_its": 4 * m},
                                ms, ts, {"status": info.status, "its": info.its, "total_its": info.total_its,
                                         "ir_steps": info.ir_steps, "k_eff": info.k_eff, "berr_dd": berr_dd(A, x, b),
                                         "ferr_vs_xstar": ferr, "ms_factor": info.ms_factor,
                                         "ms_solve": info.ms_solve}))
        # FP64 LU on the same GPU (cuSOLVER through torch), warm median
        ms, ts, xl = timed(lambda: torch.linalg.solve(A, b), max(3, args.steps), 1)
        emit(sweep_line(args, world, f"randsvd dense n={n}, kappa_2={kappa:g}: FP64 LU solve (torch.linalg.solve, "
                                     f"cuSOLVER getrf/getrs) on the same GPU",
                        {"n": n, "kappa_2": kappa, "comparator": "fp64_lu"}, ms, ts,
                        {"berr_dd": berr_dd(A, xl, b)}))
        del A, b, xstar, xl
        torch.cuda.empty_cache()

    # ---- prolate: (bf16, fp64, dd), GCRO-DR(30, k) with k = 10 against k = 0; n = 4096 at w = 0.25
    # (numerically singular) and 0.499, and at n = 4096 and 16384 with about ten eigenvalues near zero
    # (w = 0.5 - 5 / n), where the recycle space carries the slow directions from step to step
    from synth import prolate_torch
    for np_, w in (((4096, 0.25), (4096, 0.499), (4096, 0.5 - 5.0 / 4096), (n, 0.5 - 5.0 / n))
                   if "prolate" in parts else ()):
        A = prolate_torch(np_, w, device=f"cuda:{local}")
        b = torch.from_numpy(rhs_uniform(np_, 0)).to(dev)
        for k in (10, 0):
            prm = gir.Params(uf="bf16", u="fp64", ur="dd", m=30, k=k, tau=1e-8, imax=10, target_berr=-1.0,
                             carry_mode=1, max_its=120)
            ms, ts, (x, info) = timed(solve_step(A, b, prm), args.steps, args.warmup)
            emit(sweep_line(args, world, f"prolate Toeplitz n={np_}, w={w:.7g}, b~U(0,1); u_f=bf16, u=fp64, u_r=dd; "
                                         f"GCRO-DR(30, {k}), tau=1e-8, target 2u",
                            {"n": np_, "w": w, "uf": "bf16", "u": "fp64", "ur": "dd", "m": 30, "k": k}, ms, ts,
                            {"status": info.status, "its": info.its, "total_its": info.total_its,
                             "ir_steps": info.ir_steps, "berr_dd": berr_dd(A, x, b), "ms_factor": info.ms_factor,
                             "ms_solve": info.ms_solve}))
        del A, b

    # ---- conv-diff n=10000: forward solve + adjoint (gradient) through the autograd function
    if "convdiff" in parts:
        A0 = torch.from_numpy(convdiff(100, 50.0)).to(dev)
        b0 = torch.from_numpy(rhs_uniform(10000, 4)).to(dev)
        xt = torch.from_numpy(normal_vector(10000, 5)).to(dev)
        prm = gir.Params(uf="bf16", u="fp64", ur="fp64", m=40, k=10, tau=1e-8, imax=10, target_berr=1e-15,
                         carry_mode=1)

        def fwd_bwd():
            A = A0.detach().requires_grad_(True)
            b = b0.detach().requires_grad_(True)
            x = gir.GirSolve.apply(A, b, prm)
            loss = ((x - xt) ** 2).sum()
            loss.backward()
            return x.detach(), A.grad, b.grad

        ms, ts, (x, dA, db) = timed(fwd_bwd, args.steps, args.warmup)
        # the gradient against an FP64 LU solve on the same GPU (context for the timed numbers)
        xs = torch.linalg.solve(A0, b0)
        lam = torch.linalg.solve(A0.T, 2 * (xs - xt))
        emit(sweep_line(args, world, "conv-diff 5-point upwind N=100 (n=10000), Pe=50, b~U(0,1); loss=||x-x_t||^2; "
                                     "forward BF16-LU RGMRES-IR(40,10) + adjoint solve, dA, db",
                        {"n": 10000, "uf": "bf16", "u": "fp64", "ur": "fp64", "m": 40, "k": 10}, ms, ts,
                        {"berr_dd": berr_dd(A0, x, b0),
                         "db_rel_err_vs_fp64_lu": ((db - lam).abs().max() / lam.abs().max()).item(),
                         "dA_rel_err_vs_fp64_lu": ((dA + torch.outer(lam, xs)).abs().max()
                                                   / torch.outer(lam, xs).abs().max()).item()},
                        metric="ms forward + backward (adjoint) solve, conv-diff n=10000"))
        del A0, b0, xt, x, dA, db, xs, lam
        torch.cuda.empty_cache()

    # ---- batch: 512 randsvd systems, n ~ U{256..4096}, kappa_2 = 10^U(2,8), (bf16, fp64, fp64), (30, 8):
    # the persistent kernel (one launch) and the worker-stream engine on the same systems
    if "batch" in parts:
        sizes, kappas = batch_specs(512, 256, 4096, 2.0, 8.0, seed=3)
        As, bs = [], []
        for i, (nn, kp) in enumerate(zip(sizes, kappas)):
            A = randsvd_torch(nn, kp, seed=1000 + i, device=f"cuda:{local}")
            gg = torch.Generator(device=dev)
            gg.manual_seed(5000 + i)
            As.append(A)
            bs.append(A @ torch.randn(nn, dtype=torch.float64, device=dev, generator=gg))
        prm = gir.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0,
                         carry_mode=1, max_its=4 * 30)
        peaks, peak_kind = load_peaks()
        for engine in ("auto", "streams"):
            l0 = gir.launch_count()
            ms, ts, (xs_, infos, st) = timed(lambda: gir.batch_solve(As, bs, prm, engine=engine), 1, 0)
            launches = gir.launch_count() - l0
            conv = sum(1 for i in infos if i.status == 0)
            # algorithmic bytes of the Arnoldi products: 8 n^2 per A v (the float-float halves of A)
            av_bytes = sum(8.0 * nn * nn * (i.total_its + sum(i.carry_applies[:i.ir_steps]))
                           for nn, i in zip(sizes, infos))
            gbs = av_bytes / (ms * 1e-3) / 1e9
            name = ("routed by the cost model: " + gir.batch_engine(sizes, prm)) if engine == "auto" else "worker-stream engine"
            emit(sweep_line(args, world, "batch of 512 randsvd systems, n~U{256..4096}, kappa_2=10^U(2,8), b=A x*; "
                                         f"u_f=bf16, u=u_r=fp64, RGMRES-IR(30,8), target 2u; {name}",
                            {"systems": 512, "n_total": int(sum(sizes)), "uf": "bf16", "m": 30, "k": 8,
                             "max_its": 120, "engine": gir.batch_engine(sizes, prm) if engine == "auto" else "streams"}, ms, ts,
                            {"status": st, "converged": conv, "total_its": int(sum(i.total_its for i in infos)),
                             "av_bytes": av_bytes, "av_gbs_over_batch": gbs,
                             "av_frac_of_hbm": gbs / peaks["hbm_gbs"],
                             "sum_ms_factor": float(sum(i.ms_factor for i in infos)),
                             "sum_ms_solve": float(sum(i.ms_solve for i in infos)),
                             "converged_by_kappa": {f"1e{e}-1e{e + 1}": [
                                 sum(1 for i, kp in zip(infos, kappas) if 10 ** e <= kp < 10 ** (e + 1) and i.status == 0),
                                 sum(1 for kp in kappas if 10 ** e <= kp < 10 ** (e + 1))] for e in range(2, 8)}},
                            launches=launches, metric="ms for the whole batch of 512 systems"))
            del xs_
        del As, bs
        torch.cuda.empty_cache()

    # ---- a small batch for counter captures of the persistent kernel: 24 randsvd systems,
    # n ~ U{1024..2048}, kappa_2 = 10^U(2,3) (seed 5), one launch, one CTA per system
    if "batch-small" in parts:
        rng = np.random.default_rng(5)
        sizes = [int(v) for v in rng.integers(1024, 2049, 24)]
        As, bs = [], []
        for i, nn in enumerate(sizes):
            A = randsvd_torch(nn, 10 ** rng.uniform(2, 3), seed=900 + i, device=f"cuda:{local}")
            gg = torch.Generator(device=dev)
            gg.manual_seed(77 + i)
            As.append(A)
            bs.append(A @ torch.randn(nn, dtype=torch.float64, device=dev, generator=gg))
        prm = gir.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0,
                         carry_mode=1, max_its=4 * 30)
        ms, ts, (xs_, infos, st) = timed(lambda: gir.batch_solve(As, bs, prm, engine="persistent"),
                                         max(1, args.steps), args.warmup)
        emit(sweep_line(args, world, "small batch of 24 randsvd systems, n~U{1024..2048}, kappa_2=10^U(2,3); "
                                     "u_f=bf16, u=u_r=fp64, RGMRES-IR(30,8), target 2u; one persistent launch",
                        {"systems": 24, "uf": "bf16", "m": 30, "k": 8, "max_its": 120, "engine": "persistent"},
                        ms, ts, {"status": st, "total_its": int(sum(i.total_its for i in infos))},
                        metric="ms for the whole batch of 24 systems"))
        del As, bs, xs_

    # ---- the adjoint's transposed triangular solves beside the forward ones: one forward and one
    # adjoint solve with the same factors, their phases timed by the library's trace (CUDA events on
    # the solve's stream, per call), then K timed adjoint solves without the trace
    if "adjoint" in parts:
        names = ["trsv", "trsv adjoint", "gemv", "gemv adjoint"]
        for label, A in (("conv-diff 5-point upwind N=100 (n=10000), Pe=50",
                          torch.from_numpy(convdiff(100, 50.0)).to(dev)),
                         ("randsvd n=16384, kappa_2=1e2", randsvd_torch(16384, 1e2, seed=0, device=f"cuda:{local}"))):
            nn = A.shape[0]
            b = torch.from_numpy(rhs_uniform(nn, 4)).to(dev)
            prm = gir.Params(uf="bf16", u="fp64", ur="fp64", m=40, k=10, tau=1e-8, imax=10, target_berr=1e-15)
            F = gir.Factorization(A, prm)
            F.solve(A, b)
            F.solve_adjoint(A, b)
            torch.cuda.synchronize()
            gir.trace_enable(True)
            gir.trace_select(names)
            x, info = F.solve(A, b)
            lam, ia = F.solve_adjoint(A, b)
            torch.cuda.synchronize()
            rep = gir.trace_report()
            gir.trace_enable(False)
            ms, ts, _ = timed(lambda: F.solve_adjoint(A, b), max(1, args.steps), args.warmup)
            per_call = {k: {"ms": v[0], "calls": v[1], "us_per_call": 1e3 * v[0] / max(v[1], 1)}
                        for k, v in rep.items()}
            emit(sweep_line(args, world, f"{label}, b~U(0,1); BF16 LU, RGMRES-IR(40,10); adjoint solve A^T lambda = b "
                                         "with the forward solve's factors",
                            {"n": nn, "uf": "bf16", "u": "fp64", "ur": "fp64", "m": 40, "k": 10}, ms, ts,
                            {"forward_its": info.total_its, "adjoint_its": ia.total_its, "trace": per_call,
                             "trsv_adjoint_over_forward": (per_call["trsv adjoint"]["us_per_call"]
                                                           / per_call["trsv"]["us_per_call"])},
                            metric="ms per adjoint solve (factors given)"))
            F.close()
            del A, b, x, lam
            torch.cuda.empty_cache()

    # ---- the oracle at two sizes (validates the n^3 projection of the headline's cpu_baseline)
    if rank == 0 and not args.no_cpu and "oracle" in parts:
        proj, t1, t2, expo, i1, i2 = oracle_projection(args.n, args.sample_n, args.kappa, args.uf)
        n1, n2 = args.sample_n // 2, args.sample_n
        pts = [(n1, t1, i1.paper_format()), (n2, t2, i2.paper_format())]
        emit({"metric": "oracle seconds (CPU) on randsvd kappa_2=1e2 at two sizes", "sweep": True,
              "value": t2, "unit": "s", "cpu_baseline": {"value": t2 * 1e3, "unit": "ms", "cores": os.cpu_count(),
                                                          "kind": "oracle", "sample": f"n={n2}"},
              "result": {"points": [{"n": a, "s": b, "its": c} for a, b, c in pts], "fitted_exponent": expo,
                         "projected_ms_n16384": t2 * 1e3 * (args.n / n2) ** expo, "cpu": cpu_model()}})
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--kappa", type=float, default=1e2)
    ap.add_argument("--uf", default="fp16")
    ap.add_argument("--m", type=int, default=50)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--sample-n", type=int, default=3072)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-lu", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="the measurement matrix instead of the headline: kappa_2 x u_f with the k = 0 comparator, "
                         "the FP64 LU comparator, prolate n=4096 recycling counts, conv-diff n=10000 forward + "
                         "backward, the 512-system batch and the oracle at two sizes; one JSON line per point")
    ap.add_argument("--only", default="",
                    help="with --sweep: a comma-separated subset of randsvd,prolate,convdiff,batch,oracle, or "
                         "batch-small (24 systems for counter captures of the persistent kernel) or adjoint "
                         "(the transposed triangular solves of M^-T against the forward ones, by the trace)")
    args = ap.parse_args()
    rank, world, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args, rank, world, local)

    import torch
    import paper_2201_09827_gb300 as gir
    from paper_2201_09827_gb300.shard import max_over_ranks
    from synth import randsvd_torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    peaks, peak_kind = load_peaks()

    n = args.n
    A = randsvd_torch(n, args.kappa, seed=rank, device=f"cuda:{local}")
    g = torch.Generator(device=dev)
    g.manual_seed(2 + 100 * rank)
    xstar = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    b = A @ xstar
    prm = gir.Params(uf=args.uf, u="fp64", ur="fp64", m=args.m, k=args.k, tau=1e-8, imax=10, target_berr=1e-15,
                     carry_mode=1)

    def step(Ad, bd, x):
        F = gir.Factorization(Ad, prm)
        _, info = F.solve(Ad, bd, x)
        F.close()
        return info

    def step_x(Ad, bd, p):
        F = gir.Factorization(Ad, p)
        xx, info = F.solve(Ad, bd)
        F.close()
        return xx, info

    x = torch.empty_like(b)
    for _ in range(args.warmup):
        info = step(A, b, x)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---------------- timed region (device-resident inputs) ----------------
    # CUDA events bracket only the kernels the roofline reads; events between every launch would
    # add about 4 ms to a step (measured)
    gir.trace_select(ROOFLINE_PHASES)
    gir.trace_enable(True)
    l0 = gir.launch_count()
    times, infos = [], []
    with ClockSampler(local) as clk:
        barrier()
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(A, b, x)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        barrier()
    launches = gir.launch_count() - l0
    trace = gir.trace_report()
    gir.trace_enable(False)
    gir.trace_select(None)
    clocks = clk.summary()
    # the phase breakdown: one more step, after the timed region, with every phase timed
    gir.trace_enable(True)
    step(A, b, x)
    breakdown = gir.trace_report()
    gir.trace_enable(False)

    # correctness of the timed result: backward error from a double-double residual
    r = gir.residual(A, x, b, "dd")
    eta = (r.abs().max() / (A.abs().sum(1).max() * x.abs().max() + b.abs().max())).item()
    ms = max_over_ranks(statistics.median(times), device=dev)

    # ---------------- end to end through the public API with host buffers ----------------
    # gir.solve with pinned CPU tensors: H2D of A and b, factor + solve, D2H of x, per step
    e2e = None
    if not args.no_e2e:
        Ah = A.cpu().pin_memory()
        bh = b.cpu().pin_memory()
        et = []
        for it in range(max(2, args.steps // 2) + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xh, _ = gir.solve(Ah, bh, prm)
            e1.record(stream)
            e1.synchronize()
            if it > 0:
                et.append(e0.elapsed_time(e1))
        e2e = {"value": statistics.median(et), "unit": "ms", "h2d_bytes_per_step": 8 * n * n + 8 * n,
               "d2h_bytes_per_step": 8 * n, "api": "paper_2201_09827_gb300.solve(A_host_pinned, b_host_pinned)"}
        del Ah, bh

    # ---------------- comparators on the same GPU ----------------
    def timed_steps(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts, res = [], None
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), res

    comparators = {}
    fp64_lu_ms = None
    if not args.no_fp64_lu and rank == 0:
        # FP64 LU solve (cuSOLVER getrf/getrs through torch), warm median of 3
        fp64_lu_ms, xl = timed_steps(lambda: torch.linalg.solve(A, b), 3, 1)
        comparators["fp64_lu"] = {"ms": fp64_lu_ms, "api": "torch.linalg.solve (cuSOLVER), warm median of 3"}
        del xl
    if rank == 0 and not args.no_comparators:
        # GMRES-IR (k = 0) on the same system
        prm0 = gir.Params(uf=args.uf, u="fp64", ur="fp64", m=args.m, k=0, tau=1e-8, imax=10, target_berr=1e-15,
                          carry_mode=1)
        ms0, (_, i0) = timed_steps(lambda: step_x(A, b, prm0), 3, 1)
        comparators["gmres_ir_same_system"] = {"ms": ms0, "its": i0.its, "total_its": i0.total_its,
                                               "status": i0.status, "m": args.m, "k": 0, "uf": args.uf}
        # the same system with a BF16 LU (not one of the paper's formats; eight bits of significand)
        if args.uf != "bf16":
            prm_b = gir.Params(uf="bf16", u="fp64", ur="fp64", m=args.m, k=args.k, tau=1e-8, imax=10,
                               target_berr=1e-15, carry_mode=1)
            msb, (_, ib) = timed_steps(lambda: step_x(A, b, prm_b), 3, 1)
            comparators["bf16_same_system"] = {"ms": msb, "its": ib.its, "total_its": ib.total_its,
                                               "status": ib.status, "m": args.m, "k": args.k, "uf": "bf16"}
        # recycling where the preconditioned operator has a few outlying eigenvalues: prolate
        # Toeplitz with about ten eigenvalues near zero (w = 0.5 - 5/n), (bf16, fp64, dd), m = 30
        from synth import prolate_torch
        wp = 0.5 - 5.0 / n
        Ap = prolate_torch(n, wp, device=f"cuda:{local}")
        gp = torch.Generator(device=dev)
        gp.manual_seed(0)
        bp = torch.rand(n, dtype=torch.float64, device=dev, generator=gp)
        rec = {"workload": f"prolate Toeplitz n={n}, w=0.5-5/n={wp:.7f}, b~U(0,1); u_f=bf16, u=fp64, u_r=dd, "
                           f"m=30, tau=1e-8, target 2u"}
        for kk in (10, 0):
            prm_p = gir.Params(uf="bf16", u="fp64", ur="dd", m=30, k=kk, tau=1e-8, imax=10, target_berr=-1.0,
                               carry_mode=1, max_its=120)
            msp, (_, ip) = timed_steps(lambda: step_x(Ap, bp, prm_p), 3, 1)
            rec[f"k{kk}"] = {"ms": msp, "its": ip.its, "total_its": ip.total_its, "status": ip.status}
        comparators["prolate_recycling"] = rec
        del Ap, bp
        torch.cuda.empty_cache()

    # ---------------- roofline of the dominant kernel ----------------
    # Phases are kernel launches timed by CUDA events on their own streams inside the library;
    # "minv" and "cycle close" wrap several kernels and are not candidates.
    roof, others = None, []
    if trace:
        cands = sorted(((v[0], k) for k, v in trace.items() if phase_work(k, args, v[1]) is not None), reverse=True)
        for i, (tot, k) in enumerate(cands[:4]):
            r = roofline_for(k, trace[k][0], trace[k][1], args, peaks, peak_kind)
            if i == 0:
                roof = r
            else:
                others.append(r)
    phase_ms = {k: round(v[0], 3) for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1][0])}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_json(n, args.sample_n, args.kappa, args.uf)

    if rank == 0:
        last = infos[-1]
        out = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_json(args, world),
               "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
               "result": {"status": last.status, "its": last.its, "total_its": last.total_its,
                          "ir_steps": last.ir_steps, "berr_dd": eta, "ms_factor": last.ms_factor,
                          "ms_solve": last.ms_solve, "times_ms": times},
               "fp64_lu_ms": fp64_lu_ms, "comparators": comparators, "phase_ms_per_step": phase_ms,
               "roofline_next": others,
               "timing_note": ("roofline kernels timed by CUDA events inside the timed region (phases "
                               + ", ".join(ROOFLINE_PHASES) + "); phase_ms_per_step from one extra "
                               "step after it with every phase timed")}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

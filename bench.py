#!/usr/bin/env python3
"""Benchmark of the QTT Fokker-Planck time stepper on GB300.

Metric: MPS time-steps/s of the large workload (2^8 points per dimension,
N = 40 QTT sites, 2^40 grid cells, chi_max = 128, Heun RK2), with the state
resident in HBM when the timed region starts.  One PDF per GPU: with
--gpus N every rank steps its own independent PDF (replicas, weak scaling;
the method has no data-parallel exchange).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

--impl reference times the CPU finite-difference oracle on the host cores
(bounded sample of the same workload, extrapolated by cell count; the full
2^40-cell grid needs 8 TiB per array).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload  # noqa: E402

METRIC = "MPS time-steps/s at chi=128 vs plain FP64 GPU path; rel-L2 vs FP64 oracle"
FALLBACK_BF16_TFLOPS = 1900.0  # used only when MEASURED_PEAKS.json is absent
LATE_STEPS = 10  # steps timed after the last accuracy point
ACCURACY_STEPS = (25, 100)  # step counts at which every form is compared with the FP64 path
TIMING_LAUNCHES, TIMING_TC_ISSUED = 18, 19  # positions in OBS_TIMINGS after the 6 classes x 3


def measured_peaks():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}
ORACLE_SAMPLE_BITS = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", default="large", choices=list(workload.WORKLOADS))
    ap.add_argument("--precision", default="bf16x10", choices=list(workload.PRECISIONS),
                    help="contraction arithmetic of the timed form (the FP64 path is timed beside it)")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the plain FP64 path beside the form")
    ap.add_argument("--also", default="bf16x3,fp32,tf32",
                    help="other reduced forms timed and compared with the FP64 path (comma-separated)")
    ap.add_argument("--batch", type=int, default=256,
                    help="instances of the batched configuration stepped together (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=30, help="timed steps of the batched configuration")
    ap.add_argument("--adjoint-steps", type=int, default=workload.ADJOINT["steps"],
                    help="Heun steps of the timed gradient (qtt_grad) on the adjoint configuration (0: skip)")
    ap.add_argument("--config2-seeds", type=int, default=4,
                    help="seeds of the 2^6-point, chi 64, 200-step comparison of the forms (0: skip)")
    ap.add_argument("--no-config1", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, smax, reasons = [], None, set()
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu():
    """nproc and the CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    return os.cpu_count() or 1, model


def oracle_sample_all_cores(wl: str, nsteps: int = 1, procs: int | None = None):
    """The oracle's throughput with every host core busy: one single-thread
    oracle process per core, each timing nsteps steps of its own copy of the
    2^(5*ORACLE_SAMPLE_BITS)-cell sample, started together.  Returns (procs,
    mean seconds per step per process)."""
    procs = procs or (os.cpu_count() or 1)
    code = oracle_code(wl, 0, nsteps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    times = []
    for pr in ps:
        out, _ = pr.communicate()
        if pr.returncode == 0:
            times.extend(json.loads(out.strip().splitlines()[-1])["times"])
    return procs, (statistics.mean(times) if times else float("nan"))


def oracle_code(wl: str, seed: int, nsteps: int) -> str:
    return f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import oracle, workload
p = workload.make_params({wl!r}, seed={seed})
dt = p["dt"]
p["bits"] = [{ORACLE_SAMPLE_BITS}] * 5
p["dt"] = dt
g = oracle.make_grid(p["bits"])
u = oracle.velocity_field(p, g)
f = oracle.initial_pdf(p, g)
ts = []
for _ in range({nsteps}):
    t0 = time.perf_counter()
    f = oracle.rk2_step(f, g, u, p)
    ts.append(time.perf_counter() - t0)
print(json.dumps(dict(times=ts, norm=float(f.sum()))))
"""


def oracle_sample(wl: str, seed: int = 0, nsteps: int = 1):
    """Times nsteps RK2 steps of the CPU oracle on a 2^(5*ORACLE_SAMPLE_BITS)-cell
    grid of the workload (same coefficients, velocity, initial condition and dt),
    in a child process pinned to one thread.  Returns seconds per step."""
    code = oracle_code(wl, seed, nsteps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["times"]


def roofline_traffic():
    """DRAM bytes per launch of the tensor-core GEMM from the committed ncu
    summary, when it was taken on the current kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "tc_gemm_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        with open(os.path.join(ROOT, "paper_2407_09169_gb300", "csrc", "gemm_tc.cu"), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None
    return rec.get("dram_bytes_per_launch") if rec.get("gemm_tc_sha16") == sha else None


def truncate_vjp_flops(r, s, k):
    """Algorithmic FP64 flops of one qtt_truncate_vjp call: 2 M N K for every
    product the pass issues (bonds r of X, s of the cotangent, kept counts
    k[1..N-1]), and per cut the eigen-decomposition's Householder
    tridiagonalisation (4/3 n^3) and back-transformation (2 n^3)."""
    N = len(r) - 1
    g = 2 * r[N - 1] * r[N - 1] * 2
    for n in range(N - 1, 1, -1):
        g += 2 * (2 * r[n - 1]) * r[n] * r[n] + 2 * r[n - 1] * r[n - 1] * (2 * r[n])
    for n in range(1, N):
        g += 2 * r[n] * r[n] * k[n]
        g += 2 * r[n - 1] * (2 * s[n]) * s[n - 1] + 2 * r[n] * s[n] * (2 * r[n - 1]) + 2 * r[n] * s[n] * r[n]
    g += 2 * r[N - 1] * 2 * s[N - 1] + 2 * s[N - 1] * r[N - 1] * 2
    for n in range(2, N):
        g += 2 * (2 * r[n - 1]) * r[n] * r[n]
    for n in range(N - 1, 1, -1):
        g += 2 * (2 * s[n - 1]) * r[n] * s[n] + 2 * s[n - 1] * r[n - 1] * (2 * r[n])
    for n in range(1, N):
        rl, rr, sr, kk = r[n - 1], r[n], s[n], k[n]
        nd = rr - kk
        g += 2 * (2 * rl) * rr * sr + 2 * rr * rr * (2 * rl) + 2 * rr * rr * kk
        if kk and nd:
            g += 2 * nd * rr * rr + 2 * nd * kk * rr + 2 * rr * kk * nd + 2 * rr * rr * kk
        g += 2 * (2 * rl) * rr * rr + 2 * rr * rr * (2 * rl) + 2 * (2 * rl) * rr * rr
    e = sum((4.0 / 3.0) * r[n] ** 3 + 2.0 * r[n] ** 3 for n in range(1, N))
    return float(g), float(e)


def truncate_vjp_bench(q, torch, stream, nsites, ell, chi, fp64_peak, calls=3):
    """Times qtt_truncate_vjp at a step's sizes (inputs from
    workload.make_truncation_trains: X of bond ell in the zip-up's
    left-orthonormal form, the cotangent of bond chi); CUDA events on the
    bench stream around `calls` calls after one untimed call."""
    r, xh, sb, yh = workload.make_truncation_trains(nsites, ell, chi)
    xd = torch.from_numpy(xh).cuda()
    yd = torch.from_numpy(yh).cuda()
    ro = [1] + [2 * v for v in r[1:-1]] + [1]
    cap = sum(ro[n] * 2 * ro[n + 1] for n in range(nsites))
    out = torch.empty(cap, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    _, kept = q.qtt_truncate_vjp(r, xd, sb, yd, chi, 1e-14, 0.0, out, cap, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(calls):
        q.qtt_truncate_vjp(r, xd, sb, yd, chi, 1e-14, 0.0, out, cap, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / calls
    g, e = truncate_vjp_flops(r, sb, [0] + list(kept))
    ach = (g + e) / (ms * 1e-3) / 1e12
    return {
        "config": f"{nsites} sites, X bond {ell} (random isometries, Gaussian last core), cotangent bond {chi}, "
                  f"chi {chi}, tol 1e-14, eps 0",
        "ms_per_call": ms, "kept_min": int(min(kept)), "kept_max": int(max(kept)),
        "gemm_gflop": g / 1e9, "eig_gflop": e / 1e9,
        "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": ach / fp64_peak, "peak_source": "of measured: FP64 DFMA (qtt_selftest 6, this run)"},
        "timing": f"CUDA events on the bench stream around {calls} calls after one untimed call; each call "
                  "includes its work-space allocation, one host read of the eigenvalues and a stream synchronize",
    }


def oracle_rate(seconds_per_step: float, wl: str):
    cells_sample = 2 ** (5 * ORACLE_SAMPLE_BITS)
    cells_full = 2 ** (5 * workload.WORKLOADS[wl]["bits"])
    cell_steps_per_s = cells_sample / seconds_per_step
    return cell_steps_per_s / cells_full, cell_steps_per_s


def config_for(args, p):
    return {
        "workload": f"{args.workload}: 2^{p['bits'][0]} points per dimension of f(phi1,phi2;x1,x2,x3), "
                    f"N={sum(p['bits'])} QTT sites (2^{sum(p['bits'])} cells), chi_max={p['chi_max']}, "
                    f"Heun RK2, dt={p['dt']:.4g}, Omega={p['omega']}, Da={p['da']}, gamma={p['gamma']}",
        "bits_per_dim": p["bits"][0],
        "chi_max": p["chi_max"],
        "sites": sum(p["bits"]),
        "precision": args.precision,
        "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "1 GPU",
        "l2": "per-step working set (sketch environments ~0.9 GB, operand streams) exceeds the 129 MB L2; no flush",
    }


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    p = workload.make_params(args.workload, precision=args.precision)
    ncores, cpu_model = host_cpu()
    # one oracle process per host core, each a bounded sample of the workload
    nsteps = max(1, min(args.warmup + args.steps, 3))
    procs, sps = oracle_sample_all_cores(args.workload, nsteps=nsteps, procs=ncores)
    v1, cell_rate1 = oracle_rate(sps, args.workload)
    value, cell_rate = v1 * procs, cell_rate1 * procs
    sample = (f"{procs} concurrent single-thread processes of the dense FP64 finite-difference oracle (numpy), one "
              f"per host core ({cpu_model or 'CPU model unknown'}, nproc {ncores}), each {nsteps} Heun steps on the "
              f"2^{5 * ORACLE_SAMPLE_BITS}-cell grid (2^{ORACLE_SAMPLE_BITS} points per dimension) of the same workload "
              f"({sps:.1f} s per step each); aggregate {cell_rate:.3e} cell-steps/s extrapolated by cell count to "
              f"2^{sum(p['bits'])} cells")
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(args, p),
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": procs, "kind": "oracle", "sample": sample,
                         "one_core_steps_per_s": v1, "cpu_model": cpu_model, "nproc": ncores},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ my arm
def run_mine(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2407_09169_gb300 import build as qbuild

    if rank == 0:
        qbuild.build()
    if world > 1:
        dist.barrier()
    import paper_2407_09169_gb300 as q

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = workload.make_params(args.workload, seed=rank, precision=args.precision)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- timed region: device-resident state, K steps, CUDA events on the library's stream
    ctx = q.qtt_init(p, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        ctx.step(1)
    launches0 = ctx.observe(q.OBS_TIMINGS)[TIMING_LAUNCHES]
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.observe(q.OBS_TIMINGS)[TIMING_LAUNCHES] - launches0
    ms_max = max_over_ranks(ms)
    value = args.steps * world / (ms_max / 1e3)
    scal = ctx.scalars()
    nvpp = ctx.observe(q.OBS_NVPP)[0]
    bonds = ctx.observe(q.OBS_BONDS)
    state_bytes = int(sum(bonds[n] * 2 * bonds[n + 1] for n in range(len(bonds) - 1)) * 8)
    ctx.close()

    # ---- measured FP64 peak of this GPU (DFMA and f64 mma.sync throughput probes)
    fp64_probe = [float(x) for x in q.qtt_selftest(6)[:4]]
    fp64_peak = max(fp64_probe[0], fp64_probe[1])

    # ---- per-kernel-class roofline (separate pass: CUDA events around every launch)
    roofline, classes = None, None
    if not args.no_profile and rank == 0:
        os.environ["QTT_KERNEL_TIMING"] = "1"
        cp = q.qtt_init(p, stream=stream.cuda_stream)
        os.environ.pop("QTT_KERNEL_TIMING", None)
        cp.step(1)
        t0 = cp.observe(q.OBS_TIMINGS)
        nprof = max(1, min(args.steps, 3))
        cp.step(nprof)
        t1 = cp.observe(q.OBS_TIMINGS)
        cp.close()
        names = ["gemm_f64", "qr_thin", "eig_sym", "other", "gemm_tc", "gemm_small"]
        classes = {}
        for c, nm in enumerate(names):
            launches_c = t1[3 * c] - t0[3 * c]
            ms_c = t1[3 * c + 1] - t0[3 * c + 1]
            fl_c = t1[3 * c + 2] - t0[3 * c + 2]
            classes[nm] = {"launches_per_step": launches_c / nprof, "ms_per_step": ms_c / nprof,
                           "gflop_per_step": fl_c / nprof / 1e9}
        tot = sum(v["ms_per_step"] for v in classes.values()) or 1.0
        for v in classes.values():
            v["share"] = v["ms_per_step"] / tot
        if args.precision == "fp64":
            g = classes["gemm_f64"]
            ach = g["gflop_per_step"] / (g["ms_per_step"] / 1e3) / 1e3 if g["ms_per_step"] > 0 else 0.0
            roofline = {
                "kernel": "gemm_f64 (FP64 DFMA core contractions)",
                "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak,
                "peak_source": (f"of measured: FP64 throughput probe of this run (qtt_selftest 6: DFMA "
                                f"{fp64_probe[0]:.3f}, mma.sync f64 {fp64_probe[1]:.3f} TFLOP/s; the larger)"),
                "traffic": None,
            }
        else:
            g = classes["gemm_tc"]
            issued = (t1[TIMING_TC_ISSUED] - t0[TIMING_TC_ISSUED]) / nprof
            alg = g["gflop_per_step"] * 1e9
            passes = issued / alg if alg > 0 else 1.0
            peaks = measured_peaks()
            bf16 = peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS)
            peak = bf16 / passes
            ach = g["gflop_per_step"] / (g["ms_per_step"] / 1e3) / 1e3 if g["ms_per_step"] > 0 else 0.0
            roofline = {
                "kernel": "gemm_tc (tcgen05 contractions incl. operand packing)",
                "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": (f"of measured: bf16 burst {bf16} TFLOP/s (MEASURED_PEAKS.json) / {passes:.2f} "
                                "MMA passes per algorithmic flop (mean over the step's products; TF32 passes count 2)"
                                if "bf16_tflops" in peaks else
                                f"of fallback: {FALLBACK_BF16_TFLOPS} TFLOP/s bf16 / {passes:.2f} MMA passes"),
                "traffic": roofline_traffic(),
            }
        roofline["flop_per_launch"] = g["gflop_per_step"] * 1e9 / max(g["launches_per_step"], 1)
        roofline["avg_launch_us"] = g["ms_per_step"] * 1e3 / max(g["launches_per_step"], 1)
        roofline["timing"] = ("separate eager pass after the timed region: CUDA events on the launching stream "
                              "around every launch of the class, averaged over the pass's steps")
        if args.precision != "fp64":
            # the same tensor-core GEMM (packing included) on square products that fill the GPU
            big = {}
            for n_, mode_, tfl, err_ in np.array(q.qtt_selftest(4)[:-1]).reshape(-1, 4):
                name = {3: "bf16", 0: "bf16x3"}.get(int(mode_), str(int(mode_)))
                mma_passes = 3.0 if name == "bf16x3" else 1.0
                big[f"{name}_n{int(n_)}"] = {"tflops": float(tfl), "frac": float(tfl) * mma_passes / bf16,
                                             "max_rel_err_sampled": float(err_)}
            roofline["same_kernel_large_square"] = big

    # ---- the plain FP64 GPU path at equal chi: steps/s, and every form's distance to it
    fp64_path = None
    if args.precision != "fp64" and not args.no_fp64_path:
        p64 = workload.make_params(args.workload, seed=rank, precision="fp64")
        c64 = q.qtt_init(p64, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            c64.step(1)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        c64.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        v64 = args.steps * world / (ms64 / 1e3)
        forms = [args.precision] + [x for x in args.also.split(",") if x and x != args.precision and x != "fp64"]
        fctx, fval = {}, {}
        for fm in forms:  # steps/s of each form (the headline form's is the timed value above)
            cf = q.qtt_init(workload.make_params(args.workload, seed=rank, precision=fm), stream=stream.cuda_stream)
            if fm != args.precision:
                for _ in range(args.warmup):
                    cf.step(1)
                torch.cuda.synchronize()
                e0.record(stream)
                cf.step(args.steps)
                e1.record(stream)
                torch.cuda.synchronize()
                fval[fm] = args.steps * world / (max_over_ranks(e0.elapsed_time(e1)) / 1e3)
            else:
                fval[fm] = value
            fctx[fm] = cf
        # distance to the FP64 path at equal chi after a stated number of steps,
        # beside the FP64 path's own floor (its initial condition moved by one ulp)
        acc = {fm: {} for fm in forms}
        n64 = args.warmup + args.steps
        c64u = q.qtt_init(dict(p64, ic_sigma=math.nextafter(p64["ic_sigma"], 1.0)), stream=stream.cuda_stream)
        c64u.step(n64)
        floor = {}
        for target in ACCURACY_STEPS:
            if target > n64:
                q.qtt_step_many([c64, c64u], target - n64)
                n64 = target
            floor[str(target)] = c64u.compare(c64)
            s64 = c64.scalars()
            for fm, cf in fctx.items():
                done = int(cf.scalars()["steps"])
                if target > done:
                    cf.step(target - done)
                sf = cf.scalars()
                acc[fm][str(target)] = {"rel_l2": cf.compare(c64), "d_norm_avg": sf["norm_avg"] - s64["norm_avg"],
                                        "d_mean1_avg": sf["mean1_avg"] - s64["mean1_avg"],
                                        "d_phi11_avg": sf["phi11_avg"] - s64["phi11_avg"]}
        # steps/s further into the run: the bond eigensolves take more QL
        # sweeps once the state fills its bonds (the Gram matrices of the
        # early, low-rank states deflate at once), so the step lengthens
        # along the run; timed on the same contexts right after the last
        # accuracy point
        def time_steps(c, k):
            torch.cuda.synchronize()
            e0.record(stream)
            c.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            return k * world / (max_over_ranks(e0.elapsed_time(e1)) / 1e3)

        late64 = time_steps(c64, LATE_STEPS)
        late = {fm: time_steps(cf, LATE_STEPS) for fm, cf in fctx.items()}
        for cf in fctx.values():
            cf.close()
        c64.close()
        c64u.close()
        head = acc[args.precision]
        fp64_path = {
            "value": v64, "unit": "steps/s", "ms_per_step": ms64 / args.steps, "speedup": value / v64,
            "rel_l2_vs_fp64": {k: v["rel_l2"] for k, v in head.items()},
            "fp64_one_ulp_floor": floor,
            "gate": {"rel_l2_max": 1e-5, "speedup_min": 5.0,
                     "met_at_steps": [int(k) for k, v in head.items() if v["rel_l2"] <= 1e-5 and value / v64 >= 5.0]},
            "forms": {fm: {"value": fval[fm], "unit": "steps/s", "speedup": fval[fm] / v64, "vs_fp64": acc[fm]}
                      for fm in forms},
            "later_in_run": {"window": f"steps {n64 + 1}-{n64 + LATE_STEPS} from the initial condition (CUDA events)",
                             "fp64": late64,
                             "forms": {fm: {"value": late[fm], "speedup": late[fm] / late64} for fm in forms}},
            "comparison": "each form and the FP64 path stepped from the same initial state to the stated step "
                          "counts at equal chi; relative L2 distance of the decompressed states (qtt_compare); "
                          "fp64_one_ulp_floor: the FP64 path against itself from an initial condition moved by "
                          "one ulp (ic_sigma), the reproducibility the truncation to chi leaves",
        }

    # ---- end to end through the C ABI: host params -> device, K steps, scalars read back each step
    e2e = None
    if not args.no_e2e:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ce = q.qtt_init(p, stream=stream.cuda_stream)
        for _ in range(args.steps):
            ce.step(1)
            ce.observe(q.OBS_SCALARS)
        torch.cuda.synchronize()
        dt_e2e = max_over_ranks(time.perf_counter() - t0)
        ce.close()
        e2e = {"value": args.steps * world / dt_e2e, "unit": "steps/s",
               "h2d_bytes_per_step": state_bytes // max(args.steps, 1), "d2h_bytes_per_step": 13 * 8,
               "note": "includes qtt_init (host encoding + upload of the state and operators) and a D2H read of "
                       "the 13 scalars after every step; the contraction tile and split choices are the ones the "
                       "earlier contexts of this process autotuned (first-shape tuning not in the timed region)"}

    # ---- CPU baseline (oracle), one core and every core, rank 0 at N = 1 only
    cpu = None
    parity = None
    if rank == 0 and world == 1:
        if not args.no_cpu_baseline:
            ncores, cpu_model = host_cpu()
            times = oracle_sample(args.workload, nsteps=1)
            v1, cell1 = oracle_rate(times[0], args.workload)
            procs, sps = oracle_sample_all_cores(args.workload, nsteps=1, procs=ncores)
            vall, cellall = oracle_rate(sps, args.workload)
            cpu = {"value": vall * procs, "unit": "steps/s", "cores": procs, "kind": "oracle",
                   "one_core_value": v1, "cpu_model": cpu_model, "nproc": ncores,
                   "sample": f"1 Heun step of the dense FP64 finite-difference oracle (numpy, single-thread processes) "
                             f"on the 2^{5 * ORACLE_SAMPLE_BITS}-cell grid of the same workload: one process alone "
                             f"({times[0]:.1f} s, {cell1:.3e} cell-steps/s) and {procs} processes at once, one per core "
                             f"({sps:.1f} s each, {cellall * procs:.3e} cell-steps/s together); extrapolated by cell "
                             f"count to 2^{sum(p['bits'])} cells"}
    if rank == 0 and world == 1 and not args.no_parity:
        try:
            import oracle
            ps = workload.make_params("small", precision=args.precision)
            with q.qtt_init(ps, stream=stream.cuda_stream) as cs:
                cs.step(10)
                got = cs.observe(q.OBS_DENSE)
            ref = oracle.solve(ps, 10).ravel()
            parity = {"small_workload_10_steps_rel_l2_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                      "form": args.precision}
        except Exception as ex:  # reported, never silently dropped
            parity = {"error": str(ex)}

    # ---- the 2^20-cell configuration: FP64 steps/s and distance to the oracle after 50 steps
    config1 = None
    if rank == 0 and world == 1 and not args.no_config1:
        try:
            import oracle
            pc = workload.make_params("small")
            with q.qtt_init(pc, stream=stream.cuda_stream) as cc:
                cc.step(args.warmup)
                torch.cuda.synchronize()
                e0.record(stream)
                cc.step(20)
                e1.record(stream)
                torch.cuda.synchronize()
                sps1 = 20 / (e0.elapsed_time(e1) / 1e3)
                cc.step(pc["steps"] - args.warmup - 20)
                got = cc.observe(q.OBS_DENSE)
                sc = cc.scalars()
            ref = oracle.solve(pc, pc["steps"])
            o = oracle.observables(ref, oracle.make_grid(pc["bits"]))
            config1 = {"workload": "2^4 points per dimension (2^20 cells), chi 32, FP64, 50 Heun steps",
                       "steps_per_s": sps1,
                       "rel_l2_vs_oracle": float(np.linalg.norm(got - ref.ravel()) / np.linalg.norm(ref)),
                       "d_norm_avg": sc["norm_avg"] - o["norm_avg"], "d_mean1_avg": sc["mean1_avg"] - o["mean1_avg"],
                       "d_R12": sc["R12"] - o["R12"], "d_Y12": sc["Y12"] - o["Y12"]}
        except Exception as ex:
            config1 = {"error": str(ex)}

    # ---- the 2^30-cell configuration: forms against FP64 after 200 steps, seeds 0..S-1
    config2 = None
    if rank == 0 and world == 1 and args.config2_seeds > 0:
        config2 = {"workload": "2^6 points per dimension (2^30 cells), chi 64, 200 Heun steps; fp64_one_ulp: the "
                               "FP64 path from an initial condition moved by one ulp (ic_sigma), its own floor",
                   "seeds": {}}
        for seed in range(args.config2_seeds):
            pm = workload.make_params("medium", seed=seed)
            with q.qtt_init(pm, stream=stream.cuda_stream) as cm:
                cm.step(pm["steps"])
                sm = cm.scalars()
                row = {}
                # the FP64 path's own reproducibility: its initial condition moved by one ulp
                pu = dict(pm, ic_sigma=math.nextafter(pm["ic_sigma"], 1.0))
                with q.qtt_init(pu, stream=stream.cuda_stream) as cu:
                    cu.step(pm["steps"])
                    row["fp64_one_ulp"] = {"rel_l2": cu.compare(cm)}
                for fm in ("fp32", "tf32", "bf16x10"):
                    with q.qtt_init(workload.make_params("medium", seed=seed, precision=fm),
                                    stream=stream.cuda_stream) as cf:
                        cf.step(pm["steps"])
                        sf = cf.scalars()
                        row[fm] = {"rel_l2": cf.compare(cm)}
                        for k in ("mean1_avg", "mean2_avg", "phi11_avg", "phi22_avg", "phi12_avg"):
                            row[fm]["d_" + k] = sf[k] - sm[k]
            config2["seeds"][str(seed)] = row

    # ---- batched independent PDFs (uneven grid and chi), rank 0 at N = 1 only
    batched = None
    if rank == 0 and world == 1 and args.batch > 0:
        bps = workload.make_batch_params(args.batch, seed=0, precision="fp32")
        free0 = torch.cuda.mem_get_info(dev)[0]
        t0 = time.perf_counter()
        ctxs = [q.qtt_init(bp, stream=stream.cuda_stream) for bp in bps]
        t_init = time.perf_counter() - t0
        free1 = torch.cuda.mem_get_info(dev)[0]
        q.qtt_step_many(ctxs, 3)  # eager step, the two graph captures (context by context)
        q.qtt_step_many(ctxs, 1)  # builds the batch graph
        torch.cuda.synchronize()
        launches_b0 = ctxs[0].observe(q.OBS_TIMINGS)[TIMING_LAUNCHES]
        e0.record(stream)
        q.qtt_step_many(ctxs, args.batch_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 1e3
        launches_b = ctxs[0].observe(q.OBS_TIMINGS)[TIMING_LAUNCHES] - launches_b0
        norms = [c.scalars()["norm_avg"] for c in ctxs]
        # the same contexts stepped one after another, for comparison
        nseq = max(1, min(5, args.batch_steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in ctxs:
            c.step(nseq)
        torch.cuda.synchronize()
        tseq = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        cells = sum(2.0 ** sum(bp["bits"]) for bp in bps)
        batched = {
            "instances": args.batch, "steps": args.batch_steps,
            "instance_steps_per_s": args.batch * args.batch_steps / tb,
            "ms_per_step_all_instances": tb * 1e3 / args.batch_steps,
            "precision": "fp32", "config": "Da log-U[0.1,10], Omega U[0.5,2], 2^5..2^7 points per dimension, "
                                            "chi in {16,32,64,96}, seeds 0..n-1 (workload.make_batch_params)",
            "timing": "CUDA events on the contexts' stream around one qtt_step_many call of the stated steps, each "
                      "step one launch of a graph that embeds every context's step graph; 4 untimed steps first "
                      "(eager step, graph captures, batch graph)",
            "kernel_launches_per_step": launches_b / args.batch_steps,
            "sequential_instance_steps_per_s": args.batch * nseq / tseq,
            "sequential_timing": f"host clock, each context stepped {nseq} steps alone, device synchronised",
            "init_s": t_init, "device_bytes": free0 - free1,
            "max_abs_norm_err": max(abs(v - 1.0) for v in norms), "sum_cells": cells,
        }

    # ---- discrete adjoint (qtt_grad) on the adjoint configuration, rank 0 at N = 1 only
    adjoint = None
    if rank == 0 and world == 1 and args.adjoint_steps > 0:
        pa = workload.make_adjoint_params(seed=0, precision="fp32")
        ns = args.adjoint_steps
        ck = max(1, min(workload.ADJOINT["ckpt_every"], ns))
        with q.qtt_init(pa) as ca:
            ca.grad(2, 1)  # untimed: sizes the workspaces
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Ja, ga = ca.grad(ns, ck)
            torch.cuda.synchronize()
            tg = time.perf_counter() - t0
            ca.step(2)  # the forward alone on the same context (graph capture first)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ca.step(ns)
            torch.cuda.synchronize()
            tf = time.perf_counter() - t0
        adjoint = {
            "config": "2^6 points per dimension, chi 64, FP32 form, gradient in Omega, Da, gamma, 4 velocity and "
                      "16 initial-condition amplitudes (workload.make_adjoint_params)",
            "steps": ns, "ckpt_every": ck, "n_params": int(len(ga)), "seconds": tg,
            "gradient_steps_per_s": ns / tg, "forward_steps_per_s": ns / tf, "gradient_over_forward_time": tg / tf,
            "J": Ja, "dJ_dOmega": float(ga[0]), "dJ_dDa": float(ga[1]), "dJ_dgamma": float(ga[2]),
            "timing": "host clock around one qtt_grad call (forward with checkpoints, recompute, backward) with a "
                      "device synchronize on both sides, after an untimed 2-step call",
        }

    # ---- backward of the bond truncation (qtt_truncate_vjp) at this workload's sizes, rank 0 at N = 1 only
    tvjp = None
    if rank == 0 and world == 1:
        nsites = int(sum(p["bits"]))
        tvjp = truncate_vjp_bench(q, torch, stream, nsites, int(p["chi_max"]) + int(p.get("oversample", 8)),
                                  int(p["chi_max"]), fp64_peak)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision,
            "data": "synthetic (seeded analytic velocity modes and initial PDF)",
            "config": config_for(args, p),
            "roofline": roofline, "kernel_classes": classes, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": int(launches),
            "fp64_peak": {"dfma_tflops": fp64_probe[0], "dmma_tflops": fp64_probe[1], "sms": int(fp64_probe[2]),
                          "source": "qtt_selftest 6, this run"},
            "state": {"norm_avg": scal["norm_avg"], "mean1_avg": scal["mean1_avg"], "nvpp": nvpp,
                      "discarded_weight_last_step": scal["discarded_weight"],
                      "discarded_weight_rel": scal["discarded_weight"] / scal["norm2"] if scal["norm2"] > 0 else None},
            "parity": parity, "fp64_path": fp64_path, "config1": config1, "config2": config2, "batched": batched,
            "adjoint": adjoint, "truncate_vjp": tvjp,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_mine(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

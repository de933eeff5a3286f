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
# FP64 peak of one GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.070 GHz (the unit
# count is the one that reproduces the 1.25 TFLOP/s nominal and the 1.19
# TFLOP/s measured by an FMA-throughput probe at the observed clocks).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FALLBACK_BF16_TFLOPS = 1900.0  # used only when MEASURED_PEAKS.json is absent
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
    ap.add_argument("--precision", default="bf16x3", choices=list(workload.PRECISIONS),
                    help="contraction arithmetic of the timed form (the FP64 path is timed beside it)")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the plain FP64 path beside the form")
    ap.add_argument("--also", default="fp32,tf32",
                    help="other reduced forms timed and compared with the FP64 path (comma-separated)")
    ap.add_argument("--batch", type=int, default=256,
                    help="instances of the batched configuration stepped together (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--adjoint-steps", type=int, default=20,
                    help="Heun steps of the timed gradient (qtt_grad) on the adjoint configuration (0: skip)")
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


def oracle_sample(wl: str, seed: int = 0, nsteps: int = 1):
    """Times nsteps RK2 steps of the CPU oracle on a 2^(5*ORACLE_SAMPLE_BITS)-cell
    grid of the workload (same coefficients, velocity, initial condition and dt),
    in a child process pinned to one thread.  Returns seconds per step."""
    code = f"""
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
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["times"]


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
    times = oracle_sample(args.workload, nsteps=args.warmup + args.steps)
    timed = times[args.warmup:] if len(times) > args.warmup else times
    sps = statistics.mean(timed)
    value, cell_rate = oracle_rate(sps, args.workload)
    sample = (f"{len(timed)} Heun steps of the dense FP64 finite-difference oracle (numpy, 1 thread) on the "
              f"2^{5 * ORACLE_SAMPLE_BITS}-cell grid (2^{ORACLE_SAMPLE_BITS} points per dimension) of the same "
              f"workload, extrapolated by cell count to 2^{sum(p['bits'])} cells ({cell_rate:.3e} cell-steps/s)")
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(args, p),
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample},
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
                "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (not in MEASURED_PEAKS.json)",
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
                "traffic": None,
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

    # ---- the plain FP64 GPU path at equal chi: steps/s, and the form's distance to it
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
        # advance a copy of the form to the same step count and compare at equal chi
        cf = q.qtt_init(p, stream=stream.cuda_stream)
        cf.step(args.warmup + args.steps)
        rel = cf.compare(c64)
        s64, sf = c64.scalars(), cf.scalars()
        cf.close()
        v64 = args.steps * world / (ms64 / 1e3)
        fp64_path = {
            "value": v64, "unit": "steps/s", "ms_per_step": ms64 / args.steps, "speedup": value / v64,
            "rel_l2_vs_fp64_after_steps": rel, "steps_compared": args.warmup + args.steps,
            "d_norm_avg": sf["norm_avg"] - s64["norm_avg"], "d_mean1_avg": sf["mean1_avg"] - s64["mean1_avg"],
            "d_phi11_avg": sf["phi11_avg"] - s64["phi11_avg"],
        }
        # the other reduced forms on the same workload: steps/s and distance to the FP64 path
        others = {}
        for other in [x for x in args.also.split(",") if x and x != args.precision and x != "fp64"]:
            po = workload.make_params(args.workload, seed=rank, precision=other)
            co = q.qtt_init(po, stream=stream.cuda_stream)
            for _ in range(args.warmup):
                co.step(1)
            torch.cuda.synchronize()
            e0.record(stream)
            co.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            mso = max_over_ranks(e0.elapsed_time(e1))
            so = co.scalars()
            others[other] = {"value": args.steps * world / (mso / 1e3), "unit": "steps/s",
                             "speedup": (args.steps * world / (mso / 1e3)) / v64,
                             "rel_l2_vs_fp64_after_steps": co.compare(c64),
                             "d_norm_avg": so["norm_avg"] - s64["norm_avg"]}
            co.close()
        fp64_path["other_forms"] = others
        c64.close()

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
               "h2d_bytes_per_step": state_bytes // max(args.steps, 1), "d2h_bytes_per_step": 12 * 8,
               "note": "includes qtt_init (host encoding + upload of the state and operators), per-step D2H of the 12 scalars"}

    # ---- CPU baseline (oracle) and a small-workload parity check, rank 0 at N = 1 only
    cpu = None
    parity = None
    if rank == 0 and world == 1:
        if not args.no_cpu_baseline:
            times = oracle_sample(args.workload, nsteps=1)
            v, cell_rate = oracle_rate(times[0], args.workload)
            cpu = {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"1 Heun step of the dense FP64 finite-difference oracle (numpy, 1 thread) on the "
                             f"2^{5 * ORACLE_SAMPLE_BITS}-cell grid of the same workload ({times[0]:.1f} s), "
                             f"extrapolated by cell count to 2^{sum(p['bits'])} cells ({cell_rate:.3e} cell-steps/s)"}
    if rank == 0 and world == 1 and not args.no_parity:
        try:
            import oracle
            ps = workload.make_params("small", precision=args.precision)
            with q.qtt_init(ps, stream=stream.cuda_stream) as cs:
                cs.step(10)
                got = cs.observe(q.OBS_DENSE)
            ref = oracle.solve(ps, 10).ravel()
            parity = {"small_workload_10_steps_rel_l2_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
        except Exception as ex:  # reported, never silently dropped
            parity = {"error": str(ex)}

    # ---- batched independent PDFs (uneven grid and chi), rank 0 at N = 1 only
    batched = None
    if rank == 0 and world == 1 and args.batch > 0:
        bps = workload.make_batch_params(args.batch, seed=0, precision="fp32")
        free0 = torch.cuda.mem_get_info(dev)[0]
        t0 = time.perf_counter()
        ctxs = [q.qtt_init(bp) for bp in bps]
        t_init = time.perf_counter() - t0
        free1 = torch.cuda.mem_get_info(dev)[0]
        q.qtt_step_many(ctxs, 2)  # first step eager, second captures the step graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.qtt_step_many(ctxs, args.batch_steps)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        norms = [c.scalars()["norm_avg"] for c in ctxs]
        # the same contexts stepped one after another (each synchronised), for comparison
        t0 = time.perf_counter()
        for c in ctxs:
            c.step(args.batch_steps)
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
            "timing": "host clock around qtt_step_many with a device synchronize on both sides; "
                      "2 untimed steps first (eager step, graph capture)",
            "sequential_instance_steps_per_s": args.batch * args.batch_steps / tseq,
            "init_s": t_init, "device_bytes": free0 - free1,
            "max_abs_norm_err": max(abs(v - 1.0) for v in norms), "sum_cells": cells,
        }

    # ---- discrete adjoint (qtt_grad) on the adjoint configuration, rank 0 at N = 1 only
    adjoint = None
    if rank == 0 and world == 1 and args.adjoint_steps > 0:
        pa = workload.make_adjoint_params(seed=0, precision="fp32")
        ns = args.adjoint_steps
        ck = max(1, min(workload.ADJOINT["ckpt_every"], ns // 4))
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

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision,
            "data": "synthetic (seeded analytic velocity modes and initial PDF)",
            "config": config_for(args, p),
            "roofline": roofline, "kernel_classes": classes, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": int(launches),
            "state": {"norm_avg": scal["norm_avg"], "mean1_avg": scal["mean1_avg"], "nvpp": nvpp,
                      "discarded_weight_last_step": scal["discarded_weight"]},
            "parity": parity, "fp64_path": fp64_path, "batched": batched, "adjoint": adjoint,
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

#!/usr/bin/env python
"""Benchmark: space-time dof-updates per second per V-cycle on the 2D logistic
reaction-diffusion workload (256^2 periodic grid, Nt = 256 slabs, M = 3
right-Radau nodes, 50.3M space-time dofs), FP32 cycle inside FP64 defect
correction, on one GB300 per rank.

One step = one st_vcycle call through the C ABI: FP64 residual G(U) with its
norm (one device->host read), relinearisation, one space-time V-cycle, and
the update U += e.  Inputs (U: 403 MB, workspace ~1.9 GB) are larger than the
129 MB L2, so no flush is needed between steps.

Ranks run independent replicas of the workload (each its own seeded problem,
no collective on the data path: weak scaling); value = all ranks' dofs per
step / the slowest rank's time per step.

--impl reference times the CPU oracle (slab-by-slab Newton, GMRES slab solves)
on a bounded sample of the same workload on the host cores.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time dof-updates/s per V-cycle"
UNIT = "dof/s"
WORKLOAD = dict(workload="logistic2d_256x256_Nt256_M3", grid=[256, 256], bc="periodic", Nt=256, M=3,
                nu=1e-2, rho=1.0, T=1.0, reaction="logistic rho*u*(1-u)", seed=12884,
                u0="uniform[0,1) noise smoothed by 10 neighbour-averaging passes")
FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (non-tensor) per the pool's hardware notes
KERNEL_PROBES = (("fine_residual_fp64", 0), ("level_residual_transform", 1), ("slab_jacobi", 2),
                 ("backtransform_update", 3), ("shifted_residual", 5), ("inner_restrict", 6),
                 ("prolong_add", 7), ("vcycle_graph", 4))


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (read + write) of one fine-level launch, from an ncu capture of
# `python bench.py --probe` (profiles/); valid only for the kernel source it
# was taken on (sha256 of the file that holds the kernel).
NCU_TRAFFIC = {
    # profiles/hot_kernels_logistic2d_256_Nt256_M3.md: 671.2 MB read + 177.1 MB written
    "k_inner4": {"file": "k_level4.cu", "sha256": "45927b3bd25219bec6f6b6045bdd05fc68146ab622cfaf444166009f3a195fbd", "dram_bytes": 848358912},
}


def ncu_traffic(kernel, dofs):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec:
        return None
    path = os.path.join(ROOT, "paper_2006_12883_gb300", "csrc", rec["file"])
    with open(path, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    return rec["dram_bytes"] if sha == rec["sha256"] else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle

ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import stgen
from oracle import space, system
w = json.loads({wl!r})
nslabs = int({nslabs})
shape = tuple(w["grid"])
p = system.Problem(shape=shape, bc=space.PERIODIC, nu=w["nu"], Nt=w["Nt"], M=w["M"], T=w["T"],
                   reaction=space.LOGISTIC, rho=w["rho"])
u0 = stgen.smoothed_noise(shape, w["seed"]).ravel()
out = []
for rep in range(int({reps})):
    t = time.perf_counter()
    system.solve_sequential(p, u0, nslabs=nslabs)
    out.append(time.perf_counter() - t)
print(json.dumps(out))
"""


def time_oracle(nslabs=1, reps=1):
    """Seconds per oracle solve of the first `nslabs` slabs, in a fresh
    single-threaded process (BLAS / OpenMP pinned to one thread)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, wl=json.dumps(WORKLOAD), nslabs=nslabs, reps=reps)
    r = subprocess.run([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_baseline(nslabs=1, reps=1):
    ts = time_oracle(nslabs, reps)
    Ns = WORKLOAD["grid"][0] * WORKLOAD["grid"][1]
    dofs = nslabs * WORKLOAD["M"] * Ns
    t = min(ts)
    return {"value": dofs / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"slab-by-slab Newton (GMRES slab solves) of the first {nslabs} of {WORKLOAD['Nt']} slabs "
                      f"({dofs} dofs, {t:.2f} s, best of {len(ts)})"}


# ------------------------------------------------------------------ ours

def run_ours(args):
    import torch
    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_2006_12883_gb300.build import build
        build()
    if dist:
        dist.barrier()
    import stgen
    from paper_2006_12883_gb300 import stlib

    w = WORKLOAD
    shape = tuple(w["grid"])
    u0 = stgen.smoothed_noise(shape, w["seed"] + rank).ravel()
    opts = stlib.make_opts(precision=stlib.FP32_REFINE, tol=1e-8)
    S = stlib.Solver(shape, stlib.PERIODIC, w["nu"], w["Nt"], w["M"], u0, T=w["T"], reaction=stlib.LOGISTIC,
                     rho=w["rho"], opts=opts)
    D = w["Nt"] * w["M"] * shape[0] * shape[1]
    U = S.zeros()
    stream = torch.cuda.current_stream()
    if args.probe:
        # each hot kernel in isolation at full size (for profiler captures)
        S.linearize(U)
        out = {}
        for name, which in KERNEL_PROBES[:-1]:
            kms, kb = S.time_kernel(which, U, iters=2)
            out[name] = {"ms": kms, "GBps": kb / (kms / 1e3) / 1e9}
        if rank == 0:
            print(json.dumps({"mode": "probe", "kernels": out}), flush=True)
        S.close()
        return
    for _ in range(args.warmup):
        S.vcycle(U)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    norms = []
    for _ in range(args.steps):
        norms.append(S.vcycle(U))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * D / (ms / 1e3)
    if args.only_steps:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms,
                              "mode": "only-steps (profiling run)"}), flush=True)
        S.close()
        return

    # e2e through the C ABI with host buffers (H2D + D2H of U inside every step)
    Uh = torch.zeros(S.field_shape, dtype=torch.float64).pin_memory()
    for _ in range(2):
        S.vcycle(Uh)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.vcycle(Uh)
    torch.cuda.synchronize()
    ms_e2e = (time.perf_counter() - t0) * 1e3 / args.steps
    if dist:
        t = torch.tensor([ms_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e = {"value": world * D / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": D * 8,
           "d2h_bytes_per_step": D * 8 + 8}

    stats = S.stats()
    # per-kernel live timings (CUDA events on the library's launching stream)
    kernels = {}
    for name, which in KERNEL_PROBES:
        kms, kb = S.time_kernel(which, U, iters=max(5, args.steps // 2))
        kernels[name] = {"ms": kms, "bytes": kb, "GBps": (kb / (kms / 1e3) / 1e9) if kb else None}
    hbm, src = measured_peaks()
    # dominant kernel (largest share of the cycle's time in the ncu launch
    # list): the fine-level Jacobi sweep of the shifted slab systems, fused with
    # the back-transform and the block-Jacobi update; HBM bound
    k = kernels["slab_jacobi"]
    roofline = {"bound": "hbm", "kernel": "k_inner4<2,3,1>: fine-level Jacobi sweep + back-transform + update",
                "achieved": k["GBps"], "peak": hbm, "unit": "GB/s", "frac": k["GBps"] / hbm,
                "traffic": ncu_traffic("k_inner4", D),
                "peak_source": f"{src} copy bandwidth (burst; kernel timed alone)",
                "bytes_per_dof": k["bytes"] / D}
    kf = kernels["fine_residual_fp64"]
    fine_residual = {"kernel": "k_residual_ff: FP64-accurate residual in double-float arithmetic",
                     "ms": kf["ms"], "GBps": kf["GBps"], "frac_of_hbm": kf["GBps"] / hbm,
                     "note": "issue bound on the FP32/integer pipes (double-float emulation of FP64)"}
    fp32_kernels = {n: {"GBps": kernels[n]["GBps"], "frac_of_" + src + "_hbm": kernels[n]["GBps"] / hbm}
                    for n in ("level_residual_transform", "slab_jacobi", "shifted_residual", "inner_restrict",
                              "prolong_add")}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        for name, prec in (("fp32_refine", stlib.FP32_REFINE), ("fp64", stlib.FP64)):
            S2 = stlib.Solver(shape, stlib.PERIODIC, w["nu"], w["Nt"], w["M"], u0, T=w["T"],
                              reaction=stlib.LOGISTIC, rho=w["rho"],
                              opts=stlib.make_opts(precision=prec, tol=1e-8, max_iters=100))
            V = S2.zeros()
            S2.solve(V)  # warm (graph capture)
            V.zero_()
            torch.cuda.synchronize()
            info = S2.solve(V)
            extras["time_to_1e-8_" + name] = {"seconds": info["seconds"], "iterations": info["iterations"],
                                              "rel_residual": info["rel_residual"]}
            S2.close()
        # SDC sweep throughput on the same workload
        S3 = stlib.Solver(shape, stlib.PERIODIC, w["nu"], w["Nt"], w["M"], u0, T=w["T"],
                          reaction=stlib.LOGISTIC, rho=w["rho"], opts=stlib.make_opts())
        V = S3.zeros()
        S3.sdc_sweep(V, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S3.sdc_sweep(V, 5)
        torch.cuda.synchronize()
        extras["sdc_sweep_dof_per_s"] = D * 5 / (time.perf_counter() - t0)
        S3.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = oracle_baseline(nslabs=4, reps=1)
        except Exception as ex:  # the GPU number stands without it
            cpu = {"error": str(ex)[:200]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": dict(WORKLOAD, dofs=D, precision="fp32 cycle + fp64 residual/update",
                               parallelism=f"replicas{world}", l2="inputs larger than L2 (no flush)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": stats["launches_per_vcycle"] * args.steps,
                "clocks": clk, "kernels": kernels, "fp32_kernels_hbm": fp32_kernels,
                "fine_residual": fine_residual,
                "final_rel_residual": norms[-1] / (math.sqrt(w["M"]) * float((u0 ** 2).sum()) ** 0.5),
                "extras": extras, "stats": stats}
        print(json.dumps(line), flush=True)
    S.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    if rank != 0:
        return
    ts = time_oracle(nslabs=1, reps=args.warmup + args.steps)
    timed = ts[args.warmup:]
    Ns = WORKLOAD["grid"][0] * WORKLOAD["grid"][1]
    dofs = WORKLOAD["M"] * Ns
    t = sum(timed) / len(timed)
    value = dofs / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, dofs=WORKLOAD["Nt"] * dofs, parallelism="cpu oracle, 1 thread"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: Newton (GMRES slab solves) on slab 1 of "
                                       f"{WORKLOAD['Nt']} ({dofs} dofs)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true", help="warm-up and timed steps only (profiling)")
    ap.add_argument("--probe", action="store_true", help="launch each hot kernel alone (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

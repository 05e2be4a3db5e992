#!/usr/bin/env python
"""Benchmark: space-time dof-updates per second per V-cycle on the 2D logistic
reaction-diffusion workload at full size (1024^2 periodic grid, Nt = 1024
slabs, M = 5 right-Radau nodes: 5.37e9 space-time dofs, U alone 43 GB in
FP64), FP32 cycle inside FP64 defect correction, on one GB300 per rank.  The
same workload at M = 3 (3.22e9 dofs) is reported beside it under "extras".

One step = one st_vcycle call through the C ABI: FP64-accurate residual G(U)
with its norm (one device->host read), relinearisation, one space-time
V-cycle, and the update U += e.  Inputs are far larger than the 129 MB L2, so
no flush is needed between steps.

Ranks run independent replicas of the workload (each its own seeded problem,
no collective on the data path: weak scaling); value = all ranks' dofs per
step / the slowest rank's time per step.

--impl reference times the CPU oracle on the host cores, single-threaded:
each step is one evaluation of the collocation residual (Eq. 2.3 with the
slab coupling of Eq. 3.4) over the first K slabs of the same workload (one
update of every dof those slabs hold), K chosen so that a step takes about a
second.
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
NOISE = "uniform[0,1) noise smoothed by 10 neighbour-averaging passes"
WORKLOADS = {
    # 2D logistic, 256^2 periodic, 256 slabs, 3 nodes (50.3M dofs)
    "logistic2d_256": dict(workload="logistic2d_256x256_Nt256_M3", grid=[256, 256], bc="periodic", Nt=256, M=3,
                           nu=1e-2, rho=1.0, T=1.0, reaction="logistic", seed=12884, u0=NOISE),
    "heat1d_63": dict(workload="heat1d_dirichlet63_Nt16_M2", grid=[63], bc="dirichlet", Nt=16, M=2, nu=1.0,
                      rho=0.0, T=1.0, reaction="none", seed=0, u0="sin(pi x) + 0.5 sin(3 pi x)"),
    "logistic2d_1024_m3": dict(workload="logistic2d_1024x1024_Nt1024_M3", grid=[1024, 1024], bc="periodic",
                               Nt=1024, M=3, nu=1e-2, rho=1.0, T=1.0, reaction="logistic", seed=12885, u0=NOISE),
    "logistic2d_1024_m5": dict(workload="logistic2d_1024x1024_Nt1024_M5", grid=[1024, 1024], bc="periodic",
                               Nt=1024, M=5, nu=1e-2, rho=1.0, T=1.0, reaction="logistic", seed=12885, u0=NOISE),
    "cubic3d_128": dict(workload="cubic3d_128x128x128_Nt128_M3", grid=[128, 128, 128], bc="periodic", Nt=128, M=3,
                        nu=5e-3, rho=2.0, T=1.0, reaction="cubic", seed=12886,
                        u0="8 periodic Gaussian bumps, sigma 0.05, amplitude 1"),
    "logistic2d_512": dict(workload="logistic2d_512x512_Nt512_M3", grid=[512, 512], bc="periodic", Nt=512, M=3,
                           nu=1e-2, rho=1.0, T=1.0, reaction="logistic", seed=12887, u0=NOISE),
    # a small case of the M = 5 kernel instances (1.3e8 dofs, inputs above L2, ~7 GB on the device) for
    # profiler captures
    "logistic2d_512_m5_nt96": dict(workload="logistic2d_512x512_Nt96_M5", grid=[512, 512], bc="periodic", Nt=96,
                                   M=5, nu=1e-2, rho=1.0, T=96 / 1024, reaction="logistic", seed=12885, u0=NOISE),
}
DEFAULT_CONFIG = "logistic2d_1024_m5"
WORKLOAD = WORKLOADS[DEFAULT_CONFIG]


def make_u0(w, rank=0):
    import stgen
    shape = tuple(w["grid"])
    if w["bc"] == "dirichlet":
        return stgen.sine_modes(shape[0])
    if w["reaction"] == "cubic":
        return stgen.gaussian_bumps(shape, w["seed"] + rank).ravel()
    return stgen.smoothed_noise(shape, w["seed"] + rank).ravel()


def make_solver(stlib, w, u0, **opts):
    bc = {"periodic": stlib.PERIODIC, "dirichlet": stlib.DIRICHLET}[w["bc"]]
    rx = {"none": stlib.NONE, "logistic": stlib.LOGISTIC, "cubic": stlib.CUBIC}[w["reaction"]]
    return stlib.Solver(tuple(w["grid"]), bc, w["nu"], w["Nt"], w["M"], u0, T=w["T"], reaction=rx,
                        rho=w["rho"], opts=stlib.make_opts(**opts))


HBM_DATASHEET_GBS = 7900.0  # GB300 HBM3e, vendor figure (context beside the measured copy bandwidth)
KERNEL_PROBES = (("fine_residual_fp64", 0), ("level_residual_transform", 1), ("slab_jacobi", 2),
                 ("backtransform_update", 3), ("shifted_residual", 5), ("inner_restrict", 6),
                 ("prolong_add", 7), ("slab_jacobi_plain", 8), ("update", 9), ("two_sweeps", 10),
                 ("resid_restrict", 11), ("two_sweeps_update", 12), ("vcycle_graph", 4))


def reduce_max(x, dist, device):
    """Maximum of a per-rank float over all ranks (x itself without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, dofs_per_rank, ms_per_step):
    """Whole-job throughput: every rank's dofs per step over the slowest rank's time."""
    return world * dofs_per_rank / (ms_per_step / 1e3)


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


# DRAM bytes (read + write) per space-time dof of one level-0 launch of the
# roofline kernel, from one ncu capture of `python bench.py --probe` on a
# smaller workload of the same kernel instance (its traffic grows in
# proportion to the dofs: every array is streamed once); scaled to a full
# launch by the dofs it processes.  Valid only for the kernel source it was
# taken on (sha256 of the file that holds the kernel).
NCU_TRAFFIC = {
    # k_sweep2<5, 8, 0> on 512^2 x 96 slabs x M = 5 (125.8M dofs): 1610.78 MB read + 476.65 MB written per
    # launch (the probe's two timed launches)
    "k_sweep2<5, 8, 0>": {"file": "k_sweep2.cu",
                          "sha256": "a9cc179b363433806c939574ba174a042f5c6a81725743f8fb2f46b647887b4c",
                          "dram_bytes_per_dof": (1610694400 + 476702464 + 1610873088 + 476605696) / 2 / 125829120},
    # k_sweep2<5, 8, 1> (with the update of U) on the same case: 2617.33 MB read + 968.78 MB written per launch
    "k_sweep2<5, 8, 1>": {"file": "k_sweep2.cu",
                          "sha256": "a9cc179b363433806c939574ba174a042f5c6a81725743f8fb2f46b647887b4c",
                          "dram_bytes_per_dof": (2617355264 + 968940032 + 2617312768 + 968617728) / 2 / 125829120},
}


def ncu_traffic(kernel, dofs):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec:
        return None
    path = os.path.join(ROOT, "paper_2006_12883_gb300", "csrc", rec["file"])
    with open(path, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    return rec["dram_bytes_per_dof"] * dofs if sha == rec["sha256"] else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle

# One oracle residual evaluation over the first K slabs, timed in a fresh
# single-threaded process.  The iterate is u0 on every node plus seeded noise
# of amplitude 0.1 (any iterate costs the same).
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import stgen
from oracle import space, system
w = json.loads({wl!r})
K = int({nslabs})
shape = tuple(w["grid"])
bc = dict(periodic=space.PERIODIC, dirichlet=space.DIRICHLET)[w["bc"]]
rx = dict(none=space.NONE, logistic=space.LOGISTIC, cubic=space.CUBIC)[w["reaction"]]
dt = w["T"] / w["Nt"]
p = system.Problem(shape=shape, bc=bc, nu=w["nu"], Nt=K, M=w["M"], T=K * dt, reaction=rx, rho=w["rho"])
if w["bc"] == "dirichlet":
    u0 = stgen.sine_modes(shape[0])
elif w["reaction"] == "cubic":
    u0 = stgen.gaussian_bumps(shape, w["seed"]).ravel()
else:
    u0 = stgen.smoothed_noise(shape, w["seed"]).ravel()
U = u0[None, None, :] + stgen.random_field((K, p.M, p.Ns), 4242, 0.1)
p.L
out = []
for rep in range(int({reps})):
    t = time.perf_counter()
    system.residual(p, U, u0)
    out.append(time.perf_counter() - t)
print(json.dumps(out))
"""


def oracle_slabs(w, seconds=1.0, rate=2.5e7):
    """K: how many of the workload's slabs one oracle residual step covers, so
    that a step takes about `seconds` at about `rate` dof/s on one core."""
    per_slab = w["M"] * int(math.prod(w["grid"]))
    return int(max(1, min(w["Nt"], round(seconds * rate / per_slab))))


def host_info():
    """The host's core count and CPU model (the oracle's machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform
    return {"host_nproc": os.cpu_count(), "host_cpu": model or platform.processor() or platform.machine(),
            "host_arch": platform.machine()}


def time_oracle(w, nslabs=1, reps=1):
    """Seconds per oracle residual evaluation over the first `nslabs` slabs,
    in a fresh process pinned to one core (BLAS / OpenMP on one thread)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, wl=json.dumps(w), nslabs=nslabs, reps=reps)
    cmd = [sys.executable, "-c", code]
    try:
        cpus = sorted(os.sched_getaffinity(0))
        if cpus:
            cmd = ["taskset", "-c", str(cpus[-1])] + cmd
    except Exception:
        pass
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=1500)
    if r.returncode != 0 and cmd[0] == "taskset":
        r = subprocess.run(cmd[3:], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           timeout=1500)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(w, K, n):
    return (f"oracle residual G(U) (Eq. 2.3 + slab coupling, numpy FP64) over the first {K} of {w['Nt']} slabs "
            f"({K * w['M'] * int(math.prod(w['grid']))} dofs), {n} evaluation(s); one evaluation = one update "
            f"of each of those dofs")


def oracle_baseline(w, reps=12):
    """cpu_baseline: the oracle's residual-evaluation throughput (dof/s), best of
    `reps` evaluations over the first K slabs (about 10-15 s of one core)."""
    K = oracle_slabs(w)
    ts = time_oracle(w, K, reps)
    dofs = K * w["M"] * int(math.prod(w["grid"]))
    t = min(ts)
    return dict({"value": dofs / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": oracle_sample(w, K, len(ts)) + f", best {t:.3f} s"}, **host_info())


# ------------------------------------------------------------------ ours

def host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


def pinned_host(shape):
    """A pinned host tensor of doubles (pageable if pinning fails), or None
    when it would take more than half of the host's available memory."""
    import torch
    need = 8 * math.prod(shape)
    avail = host_available_bytes()
    if avail is not None and need > avail // 2:
        return None, f"skipped: {need / 1e9:.1f} GB host buffer > half of {avail / 1e9:.1f} GB available"
    try:
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).zero_(), "pinned"
    except RuntimeError:
        return torch.zeros(shape, dtype=torch.float64), "pageable (pinning failed)"


def free_device():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def timed_solve(stlib, w, u0, prec, tol=1e-8, max_iters=100):
    """Time to `tol` from the zero iterate (second solve; the first captures
    the graphs), through st_solve on a device iterate."""
    import torch
    S = make_solver(stlib, w, u0, precision=prec, tol=tol, max_iters=max_iters)
    V = S.zeros()
    S.solve(V)
    V.zero_()
    torch.cuda.synchronize()
    info = S.solve(V)
    out = {"seconds": info["seconds"], "iterations": info["iterations"], "cycles": info["cycles"],
           "rel_residual": info["rel_residual"]}
    S.close()
    del V
    free_device()
    return out


def vcycle_rate(stlib, w, u0, steps, warmup):
    """dof-updates/s per V-cycle of another workload (device iterate, CUDA events)."""
    import torch
    S = make_solver(stlib, w, u0, precision=stlib.FP32_REFINE, tol=1e-8)
    D = w["Nt"] * w["M"] * int(math.prod(w["grid"]))
    U = S.zeros()
    for _ in range(warmup):
        S.vcycle(U)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        S.vcycle(U)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    S.close()
    del U
    free_device()
    return {"value": D / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "dofs": D, "steps": steps}


def extras_small(stlib, w, u0):
    """Times to 1e-8 (both precisions), the end-to-end solve, SDC sweeps, the
    adjoint and PFASST on a workload that fits many times over."""
    import torch
    D = w["Nt"] * w["M"] * int(math.prod(w["grid"]))
    extras = {"time_to_1e-8_fp32_refine": timed_solve(stlib, w, u0, stlib.FP32_REFINE),
              "time_to_1e-8_fp64": timed_solve(stlib, w, u0, stlib.FP64)}
    extras["e2e_solve"] = e2e_solve(stlib, w, u0, D)
    S3 = make_solver(stlib, w, u0)
    V = S3.zeros()
    S3.sdc_sweep(V, 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S3.sdc_sweep(V, 5)
    torch.cuda.synchronize()
    extras["sdc_sweep_dof_per_s"] = D * 5 / (time.perf_counter() - t0)
    S3.close()
    if w["bc"] == "periodic":
        # adjoint: gradient of 1/2 h^d |u(T) - u_target|^2 w.r.t. nu, rho, u0
        S4 = make_solver(stlib, w, u0, tol=1e-8)
        S4.set_params(1.3e-2, 0.8)
        V = S4.zeros()
        S4.solve(V)
        target = V[-1, -1].reshape(-1).clone()
        S4.set_params(w["nu"], w["rho"])
        V.zero_()
        S4.solve(V)
        du0 = torch.empty_like(target)
        S4.adjoint(V, target=target, du0=du0)  # warm (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dnu, drho, ainfo = S4.adjoint(V, target=target, du0=du0)
        torch.cuda.synchronize()
        extras["adjoint_solve"] = {"seconds": time.perf_counter() - t0, "iterations": ainfo["iterations"],
                                   "rel_residual": ainfo["rel_residual"], "dPhi_dnu": dnu, "dPhi_drho": drho}
        S4.close()
    # PFASST (3 levels, M = 1 above the finest, one sweep each) to the same
    # tolerance from u0 spread over every node, on a space-bisected hierarchy
    S5 = make_solver(stlib, w, u0, tol=1e-8, max_iters=300, coarsening=stlib.COARSEN_SPACE, pfasst_levels=3)
    u0t = torch.tensor(u0, dtype=torch.float64, device="cuda").reshape(tuple(w["grid"]))
    V = u0t.expand(S5.field_shape).contiguous()
    S5.pfasst(V.clone(), raise_on_error=False)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pinfo = S5.pfasst(V, raise_on_error=False)
    torch.cuda.synchronize()
    extras["time_to_1e-8_pfasst3"] = {"seconds": time.perf_counter() - t0, "iterations": pinfo["iterations"],
                                      "status": pinfo["status"], "rel_residual": pinfo["rel_residual"]}
    S5.close()
    free_device()
    return extras


def e2e_solve(stlib, w, u0, D):
    """End to end through st_solve with a host iterate: U copied in once, the
    V-cycles to 1e-8 on the device, the solution copied back once."""
    import torch
    S = make_solver(stlib, w, u0, precision=stlib.FP32_REFINE, tol=1e-8, max_iters=100)
    Uh, kind = pinned_host(S.field_shape)
    if Uh is None:
        S.close()
        return {"skipped": kind}
    S.solve(Uh)  # warm (graph capture)
    Uh.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = S.solve(Uh)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    S.close()
    del Uh
    free_device()
    return {"value": D * info["cycles"] / t, "unit": UNIT, "seconds": t, "cycles": info["cycles"],
            "rel_residual": info["rel_residual"], "h2d_bytes": D * 8, "d2h_bytes": D * 8, "host_buffer": kind}


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
    from paper_2006_12883_gb300 import stlib

    w = WORKLOADS[args.config]
    shape = tuple(w["grid"])
    u0 = make_u0(w, rank)
    S = make_solver(stlib, w, u0, precision=stlib.FP32_REFINE, tol=1e-8)
    D = w["Nt"] * w["M"] * int(math.prod(shape))
    U = S.zeros()
    stream = torch.cuda.current_stream()
    if args.probe:
        # each hot kernel in isolation at full size (for profiler captures)
        S.linearize(U)
        out = {}
        for name, which in KERNEL_PROBES[:-1]:
            try:
                kms, kb = S.time_kernel(which, U, iters=2)
            except stlib.StError:
                continue
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
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    value = job_value(world, D, ms)
    if args.only_steps:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms,
                              "mode": "only-steps (profiling run)"}), flush=True)
        S.close()
        return

    stats = S.stats()
    # per-kernel live timings (CUDA events on the library's launching stream)
    kernels = {}
    for name, which in KERNEL_PROBES:
        try:
            kms, kb = S.time_kernel(which, U, iters=max(5, min(20, args.steps // 2)))
        except stlib.StError as err:
            kernels[name] = {"error": str(err)[:120]}
            continue
        kernels[name] = {"ms": kms, "bytes": kb, "GBps": (kb / (kms / 1e3) / 1e9) if kb else None}
    final_rel = norms[-1] / (math.sqrt(w["M"]) * float((u0 ** 2).sum()) ** 0.5)

    # e2e through the C ABI with host buffers (H2D + D2H of U inside every
    # step); the device iterate is released first (the library stages a host
    # iterate in a device copy of its own)
    del U
    free_device()
    Uh, host_kind = pinned_host(S.field_shape)
    e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": D * 8, "d2h_bytes_per_step": D * 8 + 8,
           "host_buffer": host_kind}
    if Uh is not None:
        for _ in range(2):
            S.vcycle(Uh)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            S.vcycle(Uh)
        torch.cuda.synchronize()
        ms_e2e = reduce_max((time.perf_counter() - t0) * 1e3 / args.steps, dist, "cuda")
        e2e.update(value=job_value(world, D, ms_e2e), ms_per_step=ms_e2e)
    S.close()
    del Uh
    free_device()

    hbm, src = measured_peaks()
    # dominant kernel (largest share of the step in the ncu launch list): the
    # last two Jacobi sweeps of a slab solve in one kernel, the second fused
    # with the back-transform and the damped block-Jacobi update of e (2D
    # periodic grids in whole 64 x 8 tiles), else the fused last sweep alone;
    # timed here at level 0 where it moves the most bytes; HBM bound
    d = len(w["grid"])
    two = kernels.get("two_sweeps", {}).get("GBps") is not None
    # the step's last launch: with the update of U when the step ran it there
    upd = two and stats.get("update_in_cycle") == 1 and kernels.get("two_sweeps_update", {}).get("GBps") is not None
    k = kernels["two_sweeps_update"] if upd else (kernels["two_sweeps"] if two else kernels["slab_jacobi"])
    kname = f"k_sweep2<{w['M']}, 8, {1 if upd else 0}>" if two else f"k_inner4<{d}, {w['M']}, 2>"
    what = ("two Jacobi sweeps of the shifted slab systems in one kernel, the second fused with the back-transform "
            "and update of e" if two else
            "Jacobi sweep of the shifted slab systems fused with the back-transform and update of e")
    io = ("z, y, e, cbar and U in, U out (U += e')" if upd else "z, y, e, cbar in, e out")
    roofline = {"bound": "hbm", "kernel": kname + ": level-0 " + what + (" and of U" if upd else "") + f" ({io})",
                "achieved": k.get("GBps"), "peak": hbm, "unit": "GB/s",
                "frac": (k["GBps"] / hbm) if k.get("GBps") else None,
                "traffic": ncu_traffic(kname, D),
                "peak_source": f"{src} copy bandwidth (burst; kernel timed alone)",
                "frac_of_datasheet_7900": (k["GBps"] / HBM_DATASHEET_GBS) if k.get("GBps") else None,
                "bytes_per_dof": (k["bytes"] / D) if k.get("bytes") else None}
    kf = kernels["fine_residual_fp64"]
    fine_residual = {"kernel": f"k_residual_tile<{w['M']}>: FP64-accurate residual on the FP32 pipes",
                     "ms": kf.get("ms"), "GBps": kf.get("GBps"),
                     "frac_of_hbm": (kf["GBps"] / hbm) if kf.get("GBps") else None}
    hbm_kernels = {n: {"GBps": kernels[n]["GBps"], "frac_of_" + src + "_hbm": kernels[n]["GBps"] / hbm}
                   for n in ("level_residual_transform", "slab_jacobi", "slab_jacobi_plain", "shifted_residual",
                             "inner_restrict", "prolong_add", "update") if kernels[n].get("GBps")}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        if D > 1e9:
            # full-size workloads: what fits beside nothing else in HBM
            extras["time_to_1e-8_fp32_refine"] = timed_solve(stlib, w, u0, stlib.FP32_REFINE)
            extras["e2e_solve"] = e2e_solve(stlib, w, u0, D)
            if args.config == "logistic2d_1024_m5":
                w3 = WORKLOADS["logistic2d_1024_m3"]
                u03 = make_u0(w3)
                m3 = vcycle_rate(stlib, w3, u03, steps=max(3, min(args.steps, 20)), warmup=3)
                m3["workload"] = w3["workload"]
                m3["time_to_1e-8_fp32_refine"] = timed_solve(stlib, w3, u03, stlib.FP32_REFINE)
                m3["time_to_1e-8_fp64"] = timed_solve(stlib, w3, u03, stlib.FP64)
                extras["logistic2d_1024x1024_Nt1024_M3"] = m3
        else:
            extras = extras_small(stlib, w, u0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = oracle_baseline(w)
        except Exception as ex:  # the GPU number stands without it
            cpu = {"error": str(ex)[:200]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": dict(w, dofs=D, precision="fp32 cycle + FP64-accurate residual/update",
                               parallelism=f"replicas{world}", l2="inputs larger than L2 (no flush)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": stats["launches_per_vcycle"] * args.steps,
                "clocks": clk, "kernels": kernels, "hbm_kernels": hbm_kernels,
                "fine_residual": fine_residual, "final_rel_residual": final_rel,
                "extras": extras, "stats": stats}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    if rank != 0:
        return
    w = WORKLOADS[args.config]
    K = oracle_slabs(w)
    ts = time_oracle(w, nslabs=K, reps=args.warmup + args.steps)
    timed = ts[args.warmup:]
    dofs = K * w["M"] * int(math.prod(w["grid"]))
    t = sum(timed) / len(timed)
    value = dofs / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(w, dofs=dofs, dofs_full_workload=w["Nt"] * w["M"] * int(math.prod(w["grid"])),
                           slabs_per_step=K, parallelism="cpu oracle, 1 thread"),
            "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": "each step: " + oracle_sample(w, K, 1)}, **host_info()),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The paper's 1D examples (Section 5.3 heat, Eq. 5.1 data; Section 5.4
# monodomain), N_x = 1024 (1025 vertices, Neumann), at the (M, N_t) pairs of
# its SMG tables, with the iteration counts its single-core SMG run reports.
PAPER_PAIRS = ((1, 1024), (2, 256), (3, 32), (4, 16), (5, 8))
PAPER_ITERS = {"heat": (2, 4, 4, 5, 5), "monodomain": (16, 16, 16, 16, 58)}
PAPER_SMMG_ITERS = {"heat": (None, 12, 17, 15, 18)}
# its STMG_3^5 (space and slab bisection on every level, 5 levels), single core
PAPER_STMG_ITERS = {"heat": (6, 18, 30, 30, 30)}
# its PFASST_1^3 with one slab per core (Cores = N_t); "n.c." = not converged
PAPER_PFASST_ITERS = {"heat": (7, 30, 35, 29, 22), "monodomain": (6, 8, "n.c.", "n.c.", "n.c.")}


def run_paper_tables(args):
    """One JSON line per (example, M, coarsening): Newton iterations and
    V-cycles to the paper's tolerance 1e-9 (true collocation residual relative
    to ||G(0)||, all-FP64 path), wall time of the solve, and for the heat
    equation the max error against the fully discrete closed form
    sum_k c_k R(dt rho_k)^Nt cos(k pi x) (R the Radau IIA stability function)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2006_12883_gb300.build import build
    build()
    import stgen
    from paper_2006_12883_gb300 import stlib
    n = 1025
    for ex in ("heat", "monodomain"):
        X, T, rx, rho = (1.0, 1.0, stlib.NONE, 0.0) if ex == "heat" else (10.0, 2.0, stlib.CUBIC, 5.0)
        u0 = stgen.cosine_modes(n, X) if ex == "heat" else stgen.stimulus(n, X)
        for (M, Nt), paper_it in zip(PAPER_PAIRS, PAPER_ITERS[ex]):
            for cname, coarsening, levels in (("SMG7", stlib.COARSEN_SPACE, 7), ("SMMG7", stlib.COARSEN_SPACE_NODES, 7),
                                              ("STMG7", stlib.COARSEN_SPACE_TIME, 7),
                                              ("auto", stlib.COARSEN_AUTO_MU, 32)):
                if cname == "SMMG7" and M == 1:
                    continue  # the same hierarchy as SMG7
                # STMG: the slabs are bisected down to one, as the paper's T_l^{l+1} of size N_t/2^l;
                # every level is followed by a space bisection, so the slab solves get their whole
                # inner multigrid (not three Jacobi sweeps) against the anisotropy of mu >> 1; seven
                # levels (the paper's five leave a 65-point coarse grid, beyond the dense coarse solve)
                try:
                    S = stlib.Solver((n,), stlib.NEUMANN, 1.0, Nt, M, u0, T=T, X=X, reaction=rx, rho=rho,
                                     opts=stlib.make_opts(precision=stlib.FP64, tol=1e-9, max_iters=1000,
                                                          coarsening=coarsening, max_levels=levels,
                                                          coarse_max_slabs=1 if cname == "STMG7" else 4,
                                                          smooth_inner_levels=0 if cname == "STMG7" else 1))
                except stlib.StError as err:
                    print(json.dumps({"mode": "paper_tables", "example": ex, "M": M, "Nt": Nt, "coarsening": cname,
                                      "error": str(err)}), flush=True)
                    continue
                U = S.zeros()
                S.solve(U, raise_on_error=False)  # warm-up (graph capture)
                U.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = S.solve(U, raise_on_error=False)
                torch.cuda.synchronize()
                secs = time.perf_counter() - t0
                line = {"mode": "paper_tables", "example": ex, "M": M, "Nt": Nt, "Nx": n - 1,
                        "coarsening": cname, "levels": S.num_levels(), "status": info["status"],
                        "newton_iterations": info["iterations"], "vcycles": info["cycles"],
                        "rel_residual": info["rel_residual"], "seconds": secs,
                        "paper_smg_iterations_1core": paper_it}
                if cname == "SMMG7" and ex in PAPER_SMMG_ITERS:
                    line["paper_smmg_iterations_1core"] = PAPER_SMMG_ITERS[ex][PAPER_PAIRS.index((M, Nt))]
                if cname == "STMG7" and ex in PAPER_STMG_ITERS:
                    line["paper_stmg_iterations_1core"] = PAPER_STMG_ITERS[ex][PAPER_PAIRS.index((M, Nt))]
                if ex == "heat":
                    x = stgen.coords1d(stlib.NEUMANN, n, X)
                    h = X / (n - 1)
                    tau, Q = stlib.st_collocation(M)[:2]
                    Q = np.asarray(Q).reshape(M, M)
                    dt = T / Nt

                    def R(z):
                        return 1.0 + z * (Q[-1] @ np.linalg.solve(np.eye(M) - z * Q, np.ones(M)))

                    exact = sum(a * R(dt * (2 * np.cos(k * np.pi * h) - 2) / h ** 2) ** Nt * np.cos(k * np.pi * x)
                                for k, a in ((1, 1.0), (3, 2.0), (4, 3.0)))
                    line["max_err_vs_discrete_closed_form"] = float(np.abs(U[-1, -1].cpu().numpy() - exact).max())
                print(json.dumps(line), flush=True)
                S.close()
                del U
                torch.cuda.empty_cache()
            # PFASST_1^3: three levels, M = 1 above the finest, one sweep per level
            S = stlib.Solver((n,), stlib.NEUMANN, 1.0, Nt, M, u0, T=T, X=X, reaction=rx, rho=rho,
                             opts=stlib.make_opts(precision=stlib.FP64, tol=1e-9, max_iters=1000,
                                                  coarsening=stlib.COARSEN_SPACE, pfasst_levels=3))
            start = torch.tensor(u0, dtype=torch.float64, device="cuda").expand(S.field_shape).contiguous()
            U = start.clone()
            S.pfasst(U, raise_on_error=False)
            U = start.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = S.pfasst(U, raise_on_error=False)
            torch.cuda.synchronize()
            print(json.dumps({"mode": "paper_tables", "example": ex, "M": M, "Nt": Nt, "Nx": n - 1,
                              "coarsening": "PFASST3", "status": info["status"],
                              "pfasst_iterations": info["iterations"], "rel_residual": info["rel_residual"],
                              "seconds": time.perf_counter() - t0,
                              "paper_pfasst_iterations_Nt_cores": PAPER_PFASST_ITERS[ex][PAPER_PAIRS.index((M, Nt))]}),
                  flush=True)
            S.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # several seconds of timed steps at full size, so the 200 ms clock sampler sees many samples
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true", help="warm-up and timed steps only (profiling)")
    ap.add_argument("--probe", action="store_true", help="launch each hot kernel alone (profiling)")
    ap.add_argument("--paper-tables", action="store_true",
                    help="the paper's 1D heat and monodomain examples at its (M, Nt) pairs (JSON lines)")
    args = ap.parse_args()
    if args.paper_tables:
        run_paper_tables(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

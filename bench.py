"""Benchmark of the EQP-IFT hot path on GB300.

Workload (the configuration the headline metric is quoted on): steady 2-D
Euler, DG p = 2 on 100 x 100 x 2 triangles (20,000 elements), Mach 2, k_u = 20
state modes and k_x = 4 mesh modes, rho = 1 (full assembly), FP64. One step is
one complete ROM solve: the paper's initialisation (LM on w with tau = 0) and
the joint Levenberg-Marquardt iteration to a relative optimality of 1e-8, every
assembly and line-search evaluation running in the library's kernels inside one
CUDA graph.

Timed region: K solves, each bracketed by CUDA events on the library's stream;
L2 is flushed (a 512 MB write) between steps, outside the events. value =
solves/s over all ranks (replicas: each rank solves its own queries).
e2e: the same solves through the host API (host mu in, y, z and solve info
back), wall clock with the copies inside.
roofline: the fused assembly kernel, FP64 ALU bound; achieved = algorithmic
FLOPs of the assemblies executed in the timed region / timed duration.
cpu_baseline: the FP64 oracle's solve of the same workload on the host cores.

--impl reference runs the oracle itself (the paper provides no code; the oracle
is the reference implementation here), one solve per step.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ROM solves/sec at rel. resid 1e-8 vs FP64 oracle; element R+J evals/sec"
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the fused FP64
# assembly kernel of this workload, from an ncu capture of the current kernel
# (78.90 MB + 2.57 MB); set to None when the kernel changes until it is re-taken.
FP64_ASSEMBLY_DRAM_BYTES = 81.47e6
WORKLOAD = "euler2d_p2_20000el_ku20_kx4_rho1_fp64"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); x itself
    when the job has one rank. device: where the collective's tensor lives (a CUDA
    device for NCCL, "cpu" for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling: every
    rank processes the same number of independent units)."""
    return world * units_per_rank / max_seconds


def make_workload():
    from paper_2305_15661_gb300 import workloads as W

    return W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def probe_peak(precision: int = 0) -> float:
    """Measured throughput of this GPU (TFLOP/s, best of 3) from the probe library:
    precision 0 = FP64 FMA, 1 = FP32 FMA, 2 = FP64 tensor-core MMA (m8n8k4)."""
    import ctypes

    from paper_2305_15661_gb300 import build as B

    lib = ctypes.CDLL(B.build_probe())
    lib.fma_probe.restype = ctypes.c_int
    lib.fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_double)]
    best = 0.0
    for _ in range(3):
        v = ctypes.c_double()
        if lib.fma_probe(precision, 152 * 8, 256, 4096, ctypes.byref(v)) == 0:
            best = max(best, v.value / 1e12)
    return best


def fp64_alu_peak():
    """Measured FP64 FMA throughput of this GPU (TFLOP/s) from the FMA probe."""
    return probe_peak(0)


def cuda_event_timer(stream):
    """A timer for replica_steps: runs fn between two CUDA events recorded on
    `stream` (the stream the timed kernels are launched on) and returns its
    device time in ms."""
    import torch

    def timer(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    return timer


def replica_steps(step, steps, world, device, timer, before_step=None, sync=None):
    """The timed region of one rank of a replicas-only job: a barrier and a device
    synchronisation, `steps` calls of step() each timed by timer (before_step(),
    e.g. an L2 flush, runs untimed before each), then a synchronisation and a
    barrier. Returns (per-step ms, the job's seconds = the slowest rank's total,
    the whole-job rate in steps per second over all ranks)."""
    import torch.distributed as dist

    multi = world > 1 and dist.is_available() and dist.is_initialized()
    if multi:
        dist.barrier()
    if sync:
        sync()
    ms = []
    for _ in range(steps):
        if before_step:
            before_step()
        ms.append(timer(step))
    if sync:
        sync()
    if multi:
        dist.barrier()
    total_s = max_over_ranks(sum(ms) / 1e3, device)
    return ms, total_s, whole_job_rate(steps, world, total_s)


def cpu_baseline_solve(wl, reps=1):
    import oracle as orc
    from paper_2305_15661_gb300 import workloads as W

    O = orc.Oracle.from_workload(wl)
    mu = wl.mus[0]
    wg = wl.Phi.T @ W.replicate_guess(wl, wl.U_guess)
    times = []
    res = None
    for _ in range(reps):
        t0 = time.perf_counter()
        res = O.solve(wl.Phi, wl.Psi, mu, wg, tol=1e-8)
        times.append(time.perf_counter() - t0)
    return min(times), res, orc.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = make_workload()
    for _ in range(args.warmup):
        cpu_baseline_solve(wl)
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        _, res, threads = cpu_baseline_solve(wl)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "elements": 20000, "p": 2, "k_u": 20, "k_x": 4, "tol": 1e-8},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} full FP64 oracle solves of the workload "
                                       f"({res['init_iters']}+{res['iters']} LM steps each)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _timed_assemblies(call, stream, flush, steps, warmup):
    """Median CUDA-event time (ms) of `call` on `stream`, L2 flushed before each."""
    import torch

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    timer = cuda_event_timer(stream)
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ms.append(timer(call))
    return statistics.median(ms)


def measure_fp32_assembly(wl, dev, stream, flush, steps, warmup):
    """The mixed solve's FP32 stage kernel on the benchmark workload: one fused FP32
    assembly (R_e, Jacobians, contraction) at the evaluation point, against the
    measured FP32 FMA peak."""
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel

    ctx = ift.Context.from_workload(wl, precision=ift.FP32, stream=stream.cuda_stream)
    shapes = ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
    k = wl.ku + wl.kx
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    mu, y, z = t(wl.mus[0]), t(wl.w_eval), t(wl.tau_eval)
    S, T, H, J = (torch.zeros(n, dtype=torch.float64, device=dev) for n in (wl.ku, wl.kx, k * k, 1))
    med = _timed_assemblies(lambda: ctx.reduced_residual_jacobian_dev(mu, y, z, S, T, H, J,
                                                                      stream=stream.cuda_stream),
                            stream, flush, steps, warmup)
    ctx.close()
    fl = perfmodel.flops_per_element(2, wl.p, wl.ku, wl.kx)["total"]
    ach = fl * wl.n_elems / (med / 1e3) / 1e12
    peak = probe_peak(1)
    return {"kernel": "assemble_kernel<float,Euler,p=2,JAC>", "bound": "alu", "median_ms": med,
            "achieved_tflops": ach, "peak_tflops": peak, "frac": ach / peak if peak else None,
            "peak_source": "FP32 FMA probe on this GPU (measured)", "flops_per_element": fl,
            "warps_per_cta": shapes[0]}


def measure_batched(dev, stream, flush, steps, warmup):
    """256 hyperreduced queries on the benchmark mesh (per-query weight sets of
    100-2,000 elements) solved in one graph, FP64 and mixed; plus one batched
    evaluation of all queries at a common point, timed alone, for the gather's
    bytes per second (each sampled element reads its own Phi rows and its
    neighbours' trace rows) and its FLOP rate."""
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel
    from paper_2305_15661_gb300 import workloads as W

    B = 256
    wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2, n_mu=B, mu_box=True)
    sets = W.eq_weight_sets(wl, B, seed=3)
    n_sampled = int(sum(len(e) for e, _ in sets))
    mus = torch.as_tensor(wl.mus, dtype=torch.float64, device=dev)
    y = torch.zeros((B, wl.ku), dtype=torch.float64, device=dev)
    z = torch.zeros((B, wl.kx), dtype=torch.float64, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    fl = perfmodel.flops_per_element(2, 2, wl.ku, wl.kx)["total"]
    hbm = measured_peaks().get("hbm_gbs")
    out = {"workload": "euler2d_p2_20000el_ku20_kx4_256q_rho100to2000", "queries": B,
           "sampled_elements": n_sampled, "tol": 1e-8}
    points = {}
    for name, prec in (("fp64", ift.FP64), ("mixed", ift.MIXED)):
        ctx = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream)
        ctx.set_eq_weights_batched(sets)
        shapes = ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
        info = ctx.solve_rom_batched(wl.mus)
        med = _timed_assemblies(lambda: ctx.solve_rom_batched_dev(mus, y, z, st, stream=stream.cuda_stream),
                                stream, flush, steps, 1)
        stat = np.array([i["status"] for i in info["info"]])
        conv = int((stat == 0).sum())
        row = {"ms_per_batch": med, "solves_per_s": B / (med / 1e3), "converged": conv,
               "converged_solves_per_s": conv / (med / 1e3),
               "mean_lm_iters": float(np.mean([i["init_iters"] + i["iters"] + i["fp32_iters"]
                                               for i in info["info"]])),
               "launch_shapes": list(shapes)}
        points[name] = (stat, np.concatenate([info["w"], info["tau"]], axis=1),
                        np.array([i["J"] for i in info["info"]]))
        # the gather: one batched evaluation of every query at the evaluation point
        ys = np.tile(wl.w_eval, (B, 1))
        zs = np.tile(wl.tau_eval, (B, 1))
        ev_ms = _timed_assemblies(lambda: ctx.reduced_residual_jacobian_batched(wl.mus, ys, zs), stream, flush,
                                  steps, warmup)
        word = 8 if prec == ift.FP64 else 4
        gathered = n_sampled * perfmodel.gather_bytes_per_element(2, 2, wl.ku, word)
        gbs = gathered / (ev_ms / 1e3) / 1e9
        row["gather"] = {"kernel": "assemble_batched_kernel<%s,Euler,p=2,JAC>" % ("double" if word == 8 else "float"),
                         "ms_per_evaluation": ev_ms, "gathered_bytes": gathered, "gbs": gbs,
                         "hbm_peak_gbs": hbm, "frac_of_hbm": gbs / hbm if hbm else None,
                         "achieved_tflops": n_sampled * fl / (ev_ms / 1e3) / 1e12,
                         "timed": "host call: the query points in, one batched assembly and its per-query "
                                  "reduction, S, T, H, J out"}
        out[name] = row
        ctx.close()
    s64, z64, J64 = points["fp64"]
    smx, zmx, Jmx = points["mixed"]
    both = (s64 == 0) & (smx == 0)
    out["mixed_vs_fp64"] = {
        "both_converged": int(both.sum()),
        "max_rel_dz": float(np.max(np.linalg.norm(zmx[both] - z64[both], axis=1) / np.linalg.norm(z64[both], axis=1))),
        "max_rel_dJ": float(np.max(np.abs(Jmx[both] - J64[both]) / J64[both]))}
    return out


def run_ours(args):
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ift.load()
    wl = make_workload()
    stream = torch.cuda.Stream(device=dev)
    ctx = ift.Context.from_workload(wl, tol=1e-8, stream=stream.cuda_stream)
    shapes = ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
    mu_d = torch.as_tensor(wl.mus[0], dtype=torch.float64, device=dev)
    y_d = torch.zeros(wl.ku, dtype=torch.float64, device=dev)
    z_d = torch.zeros(wl.kx, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # warm-up (also builds the solve graph)
    info = None
    for _ in range(args.warmup):
        info = ctx.solve_rom_dev(mu_d, y_d, z_d, stream=stream.cuda_stream, want_info=True)
    assert info is not None and info["status"] == 0, info
    assemblies = 1 + info["trials"]

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    with ClockSampler(local) as clocks:
        step_ms, total_s, value = replica_steps(
            lambda: ctx.solve_rom_dev(mu_d, y_d, z_d, stream=stream.cuda_stream, want_info=False), args.steps,
            world, dev, cuda_event_timer(stream), before_step=flush_l2, sync=torch.cuda.synchronize)

    # end to end through the host API: host mu in, y, z and info out
    e2e_steps = max(3, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        out = ctx.solve_rom(wl.mus[0])
    e2e_s = time.perf_counter() - t0
    assert out["status"] == 0
    e2e_value = world * e2e_steps / e2e_s
    h2d = 8 * len(wl.mus[0])
    d2h = 2160  # solver state read back for y, z and the solve info (sizeof of the device state)

    # isolated assembly timing (device pointers), for the per-launch duration
    S = torch.zeros(wl.ku, dtype=torch.float64, device=dev)
    T = torch.zeros(wl.kx, dtype=torch.float64, device=dev)
    k = wl.ku + wl.kx
    H = torch.zeros(k * k, dtype=torch.float64, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    yv = torch.as_tensor(wl.w_eval, dtype=torch.float64, device=dev)
    zv = torch.as_tensor(wl.tau_eval, dtype=torch.float64, device=dev)
    for _ in range(3):
        ctx.reduced_residual_jacobian_dev(mu_d, yv, zv, S, T, H, J, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    n_iso = 20
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(n_iso):
        ctx.reduced_residual_jacobian_dev(mu_d, yv, zv, S, T, H, J, stream=stream.cuda_stream)
    a1.record(stream)
    a1.synchronize()
    iso_ms = a0.elapsed_time(a1) / n_iso

    # the same solve in the mixed-precision form (FP32 Jacobians and contraction;
    # FP64 residual, gradient, line search, normal equations and stopping test)
    ctx_m = ift.Context.from_workload(wl, precision=ift.MIXED, tol=1e-8, stream=stream.cuda_stream)
    ctx_m.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
    ym = torch.zeros(wl.ku, dtype=torch.float64, device=dev)
    zm = torch.zeros(wl.kx, dtype=torch.float64, device=dev)
    minfo = None
    for _ in range(args.warmup):
        minfo = ctx_m.solve_rom_dev(mu_d, ym, zm, stream=stream.cuda_stream, want_info=True)
    torch.cuda.synchronize()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(args.steps):
        ctx_m.solve_rom_dev(mu_d, ym, zm, stream=stream.cuda_stream, want_info=False)
    m1.record(stream)
    m1.synchronize()
    mixed_ms = m0.elapsed_time(m1) / args.steps
    z64 = np.concatenate([y_d.cpu().numpy(), z_d.cpu().numpy()])
    zmx = np.concatenate([ym.cpu().numpy(), zm.cpu().numpy()])
    mixed = {"value": 1e3 / mixed_ms, "unit": "solves/s", "ms_per_solve": mixed_ms,
             "stages": {k: minfo[k] for k in ("fp32_iters", "fp32_trials", "init_iters", "iters", "trials", "h_evals")},
             "rel_dz_vs_fp64": float(np.linalg.norm(zmx - z64) / np.linalg.norm(z64)),
             "form": "FP32 element Jacobians and contraction to 1e-6, then FP32 H with FP64 residual, gradient and "
                     "objective to 1e-8; line search, normal equations and stopping test FP64"}
    ctx_m.close()

    fl = perfmodel.flops_per_element(2, 2, wl.ku, wl.kx)["total"]
    n_el = wl.n_elems
    # achieved over the timed region: all assemblies of the K solves / timed duration
    achieved_tf = assemblies * args.steps * fl * n_el / (sum(step_ms) / 1e3) / 1e12
    iso_tf = fl * n_el / (iso_ms / 1e3) / 1e12
    peak_tf = fp64_alu_peak()
    mma_tf = probe_peak(2)
    evals_per_s = world * assemblies * args.steps * n_el / total_s

    # the other configurations of the method, measured after the timed region
    extras = {}
    if rank == 0 and not args.no_extras:
        extras["fp32_assembly"] = measure_fp32_assembly(wl, dev, stream, flush, max(5, args.steps), 3)
        extras["batched"] = measure_batched(dev, stream, flush, 2, 3)
        extras["warmstart"] = warmstart_measurement(dev, stream, ift.MIXED, ift.CONTRACT_FP, 2048, 4096, 1500, 2, 32)

    line = None
    if rank == 0:
        launches_per_solve = 4 + 3 * assemblies
        cpu = None
        if world == 1 and not args.no_cpu:
            cpu_s, res, threads = cpu_baseline_solve(wl)
            cpu = {"value": 1.0 / cpu_s, "unit": "solves/s", "cores": threads, "kind": "oracle",
                   "sample": f"one full FP64 oracle solve of the workload ({res['init_iters']}+{res['iters']} "
                             f"LM steps, {cpu_s:.1f} s)"}
        clk = clocks.summary()
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "elements": n_el, "p": 2, "k_u": wl.ku, "k_x": wl.kx,
                           "tol": 1e-8, "l2": "flushed between steps (512 MB write)",
                           "assemblies_per_solve": assemblies, "parallelism": f"replicas{world}",
                           "launch_shapes": {"warps_per_cta": shapes[0]}},
                "element_rj_evals_per_s": evals_per_s, "mixed_precision": mixed,
                "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "roofline": {"bound": "alu", "kernel": "assemble_kernel<double,Euler,p=2,JAC>",
                             "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                             "frac": achieved_tf / peak_tf if peak_tf else None,
                             "traffic": FP64_ASSEMBLY_DRAM_BYTES,
                             "peak_source": "FP64 FMA probe on this GPU (measured)",
                             "flops_per_element": fl, "isolated_assembly_ms": iso_ms,
                             "isolated_achieved": iso_tf, "fp64_mma_probe_tflops": mma_tf},
                "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches_per_solve * args.steps}
        line.update(extras)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _precision(args):
    from paper_2305_15661_gb300 import ift

    return {"fp64": ift.FP64, "fp32": ift.FP32, "mixed": ift.MIXED, "fp32jac": ift.FP32_JACOBIAN}[args.precision]


def _contraction(args):
    from paper_2305_15661_gb300 import ift

    if args.precision == "fp64":
        return ift.CONTRACT_FP
    return {"fp": ift.CONTRACT_FP, "tf32": ift.CONTRACT_TF32, "3xtf32": ift.CONTRACT_3XTF32,
            "bf16": ift.CONTRACT_BF16}[args.contraction]


def run_assembly(args):
    """Isolated fused assemblies of the workload at its evaluation point."""
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel

    from paper_2305_15661_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    ift.load()
    if args.config == 4:  # p = 3 on 200 x 200 x 2 triangles, k_u = 40, k_x = 8
        wl = W.euler_workload(n=200, p=3, k_u=40, k_x=8, seed=4, q=args.q, curve=0.4 if args.q == 2 else 0.0)
    elif args.q == 2:  # the same p = 2 workload on curved six-node triangles
        wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2, q=2, curve=0.4)
    else:
        wl = make_workload()
    stream = torch.cuda.Stream(device=dev)
    prec = {"fp64": ift.FP64, "fp32": ift.FP32, "mixed": ift.FP32, "fp32jac": ift.FP32_JACOBIAN}[args.precision]
    ctx = ift.Context.from_workload(wl, precision=prec, stream=stream.cuda_stream, contraction=_contraction(args))
    shapes = ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval) if args.autotune else None
    k = wl.ku + wl.kx
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev)
    mu, y, z = t(wl.mus[0]), t(wl.w_eval), t(wl.tau_eval)
    S, T, H, J = (torch.zeros(n, dtype=torch.float64, device=dev) for n in (wl.ku, wl.kx, k * k, 1))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.reduced_residual_jacobian_dev(mu, y, z, S, T, H, J, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.reduced_residual_jacobian_dev(mu, y, z, S, T, H, J, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    fl = perfmodel.flops_per_element(2, wl.p, wl.ku, wl.kx)["total"]
    med = statistics.median(ms)
    print(json.dumps({"mode": "assembly", "precision": args.precision, "contraction": args.contraction,
                      "elements": wl.n_elems, "p": wl.p, "q": wl.q,
                      "k_u": wl.ku, "k_x": wl.kx, "launch_shapes": shapes,
                      "median_ms": med, "min_ms": min(ms), "element_rj_evals_per_s": wl.n_elems / (med / 1e3),
                      "achieved_tflops": fl * wl.n_elems / (med / 1e3) / 1e12, "flops_per_element": fl}))
    ctx.close()
    return 0


def run_batched(args):
    """256 parameter queries with uneven hyperreduced weight sets, solved in one graph."""
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel
    from paper_2305_15661_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    ift.load()
    if args.config == 4:  # p = 3, 80,000 elements, k_u = 40, k_x = 8, 1,024 queries
        B = 1024
        wl = W.euler_workload(n=200, p=3, k_u=40, k_x=8, seed=4, n_mu=B, mu_box=True)
        sets = W.eq_weight_sets(wl, B, seed=5)
    else:  # p = 2, 20,000 elements, k_u = 20, k_x = 4, 256 queries
        B = 256
        wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2, n_mu=B, mu_box=True)
        sets = W.eq_weight_sets(wl, B, seed=3)
    stream = torch.cuda.Stream(device=dev)
    prec = _precision(args)
    ctx = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream,
                                    contraction=_contraction(args), max_iters=args.max_iters)
    ctx.set_eq_weights_batched(sets)
    shapes = ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
    mus = torch.as_tensor(wl.mus, dtype=torch.float64, device=dev)
    y = torch.zeros((B, wl.ku), dtype=torch.float64, device=dev)
    z = torch.zeros((B, wl.kx), dtype=torch.float64, device=dev)
    st = torch.zeros(B, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    info = ctx.solve_rom_batched(wl.mus)
    for _ in range(args.warmup):
        ctx.solve_rom_batched_dev(mus, y, z, st, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve_rom_batched_dev(mus, y, z, st, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    conv = int((st == 0).sum().item())
    evals = sum(len(sets[q][0]) * (1 + info["info"][q]["trials"]) for q in range(B))
    fl = perfmodel.flops_per_element(2, wl.p, wl.ku, wl.kx)["total"]
    t = sum(ms) / 1e3
    out = {"mode": "batched", "config": args.config, "elements": wl.n_elems, "p": wl.p,
           "k_u": wl.ku, "k_x": wl.kx, "precision": args.precision, "contraction": args.contraction,
           "queries": B, "launch_shapes": shapes, "max_iters": args.max_iters,
           "converged_solves_per_s": conv * args.steps / t,
           "elements_per_query_mean": float(np.mean([len(s[0]) for s in sets])),
           "converged": conv, "ms_per_batch": 1e3 * t / args.steps,
           "solves_per_s": B * args.steps / t, "element_rj_evals_per_batch": evals,
           "achieved_tflops": evals * fl * args.steps / t / 1e12,
           "mean_iters": float(np.mean([i["init_iters"] + i["iters"] + i["fp32_iters"] for i in info["info"]])),
           "mean_fp64_iters": float(np.mean([i["iters"] for i in info["info"]]))}
    if args.compare_fp64 and prec != ift.FP64:
        # the same queries solved with FP64 assemblies throughout: converged points and objectives
        ref_ctx = ift.Context.from_workload(wl, precision=ift.FP64, tol=1e-8, stream=stream.cuda_stream,
                                            max_iters=args.max_iters)
        ref_ctx.set_eq_weights_batched(sets)
        try:
            ref_ctx.set_launch_shapes(*shapes)
        except ift.IFTError:
            pass  # the FP64 kernels do not fit these warps: keep their default shapes
        t0 = time.perf_counter()
        ref = ref_ctx.solve_rom_batched(wl.mus)
        out["fp64_batch_s"] = time.perf_counter() - t0
        ok = np.array([a["status"] == 0 and b["status"] == 0 for a, b in zip(info["info"], ref["info"])])
        z1 = np.concatenate([info["w"], info["tau"]], axis=1)[ok]
        z0 = np.concatenate([ref["w"], ref["tau"]], axis=1)[ok]
        J1 = np.array([i["J"] for i in info["info"]])[ok]
        J0 = np.array([i["J"] for i in ref["info"]])[ok]
        dz = np.linalg.norm(z1 - z0, axis=1) / np.linalg.norm(z0, axis=1)
        out["vs_fp64"] = {"both_converged": int(ok.sum()), "median_rel_dz": float(np.median(dz)),
                          "max_rel_dz": float(np.max(dz)), "max_rel_dJ": float(np.max(np.abs(J1 - J0) / J0)),
                          "fp64_mean_iters": float(np.mean([i["init_iters"] + i["iters"] for i in ref["info"]]))}
        ref_ctx.close()
    print(json.dumps(out))
    ctx.close()
    return 0


def _time_batched(ctx, stream, mus, y0, z0, y, z, st, steps):
    """CUDA-event time of `steps` batched solves from the starts (y0, z0); the
    start is copied into (y, z) before each step, outside the events."""
    import torch

    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            y.copy_(y0)
            z.copy_(z0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve_rom_batched_dev(mus, y, z, st, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def run_warmstart(args):
    """Learned warm start: 2,048 training solves by the method on the 20,000-element
    Euler mesh (p = 2, k_u = 40, k_x = 8, one shared weight set on 2% of the
    elements), a 2 -> 128 -> 128 -> 128 -> 48 GELU network trained on them by the
    library's kernels, then 4,096 batched queries started from the network, from
    the nearest training point and from the projected guess; and the plain FP64
    one-query solve of a sample of the same queries for comparison."""
    import torch

    from paper_2305_15661_gb300 import ift

    dev = torch.device("cuda", 0)
    ift.load()
    stream = torch.cuda.Stream(device=dev)
    out = {"mode": "warmstart", "precision": args.precision, "contraction": args.contraction}
    out.update(warmstart_measurement(dev, stream, _precision(args), _contraction(args), args.train_solves,
                                     args.queries, args.epochs, args.steps, args.single_sample))
    print(json.dumps(out))
    return 0


def warmstart_measurement(dev, stream, prec, contraction, n_train, n_query, epochs, steps, single_sample):
    """The measurement of run_warmstart, returned as a dict (also a key of the
    default bench line). Every start is judged by the same FP64 stopping test; the
    learned start's converged points are compared with the plain FP64 one-query
    solves of the sample queries (same tolerance, projected start)."""
    import torch

    from paper_2305_15661_gb300 import ift
    from paper_2305_15661_gb300 import workloads as W

    wl = W.euler_workload(n=100, p=2, k_u=40, k_x=8, seed=2)
    ku, kx = wl.ku, wl.kx
    rho_set = W.eq_weight_sets(wl, 1, seed=3, lo=400, hi=401)[0]
    mu_t = W.mu_box_samples(5, 1, n_train)
    mu_q = W.mu_box_samples(6, 1, n_query)
    out = {"workload": "euler2d_p2_20000el_ku40_kx8_rho400", "train_solves": n_train, "queries": n_query,
           "rho_nnz": int(len(rho_set[0])), "k_u": ku, "k_x": kx}

    # training data: the method's own solves from the projected guess
    gen = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream,
                                    contraction=contraction)
    gen.set_eq_weights_batched([rho_set] * n_train)
    out["launch_shapes"] = gen.autotune(mu_t[0], wl.w_eval, wl.tau_eval)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = gen.solve_rom_batched(mu_t)
    out["train_data_s"] = time.perf_counter() - t0
    ok = np.array([i["status"] == 0 for i in res["info"]])
    out["train_converged"] = int(ok.sum())
    y_t = np.concatenate([res["w"], res["tau"]], axis=1)[ok]
    gen.close()

    net = ift.MLP(2, 128, 3, ku + kx, seed=7, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out["train_loss"] = net.train(mu_t[ok], y_t, epochs=epochs, batch=64, lr=1e-3, seed=8)
    out["train_s"] = time.perf_counter() - t0
    out["epochs"] = epochs
    t0 = time.perf_counter()
    start_mlp = net.predict(mu_q)
    out["predict_ms"] = 1e3 * (time.perf_counter() - t0)
    net.predict_bf16(mu_q[:128])  # first call: kernel attributes and buffers
    t0 = time.perf_counter()
    start_bf16 = net.predict_bf16(mu_q)
    out["predict_bf16_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    start_nn = ift.nearest_start(mu_t[ok], y_t, mu_q, scale=1.0 / W.MU_BOX_WIDTH)
    out["nearest_ms"] = 1e3 * (time.perf_counter() - t0)

    given = ift.Context.from_workload(wl, precision=prec, tol=1e-8, lm_init=ift.INIT_GIVEN,
                                      stream=stream.cuda_stream, contraction=contraction)
    given.set_eq_weights_batched([rho_set] * n_query)
    given.set_launch_shapes(*out["launch_shapes"])
    paper = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream,
                                      contraction=contraction)
    paper.set_eq_weights_batched([rho_set] * n_query)
    paper.set_launch_shapes(*out["launch_shapes"])
    ref = paper.solve_rom_batched(mu_q)
    z_ref = np.concatenate([ref["w"], ref["tau"]], axis=1)
    J_ref = np.array([i["J"] for i in ref["info"]])
    ok_ref = np.array([i["status"] == 0 for i in ref["info"]])

    mus = torch.as_tensor(mu_q, dtype=torch.float64, device=dev)
    y = torch.zeros((n_query, ku), dtype=torch.float64, device=dev)
    z = torch.zeros((n_query, kx), dtype=torch.float64, device=dev)
    st = torch.zeros(n_query, dtype=torch.int32, device=dev)
    rows = {}
    for name, ctx, s in (("projected", paper, None), ("nearest", given, start_nn), ("mlp", given, start_mlp),
                         ("mlp_bf16", given, start_bf16)):
        if s is None:
            info = ref
            y0 = torch.zeros_like(y)
            z0 = torch.zeros_like(z)
        else:
            info = ctx.solve_rom_batched(mu_q, s[:, :ku], s[:, ku:])
            y0 = torch.as_tensor(np.ascontiguousarray(s[:, :ku]), device=dev)
            z0 = torch.as_tensor(np.ascontiguousarray(s[:, ku:]), device=dev)
        ms = _time_batched(ctx, stream, mus, y0, z0, y, z, st, steps)
        stat = np.array([i["status"] for i in info["info"]])
        its = np.array([i["init_iters"] + i["iters"] + i["fp32_iters"] for i in info["info"]])
        zf = np.concatenate([info["w"], info["tau"]], axis=1)
        both = ok_ref & (stat == 0)
        Jf = np.array([i["J"] for i in info["info"]])
        gfin = np.array([math.hypot(i["normS"], i["normT"]) for i in info["info"]])
        thr = np.array([1e-8 * max(1.0, i["g0"]) for i in info["info"]])
        row = {"ms_per_batch": statistics.median(ms), "solves_per_s": n_query / (statistics.median(ms) / 1e3),
               "converged": int((stat == 0).sum()), "mean_lm_iters": float(its.mean()),
               "max_iters": int(its.max()),
               "median_final_gradient": float(np.median(gfin)), "median_threshold": float(np.median(thr)),
               "max_rel_dz_vs_projected_start": float(np.max(np.linalg.norm(zf[both] - z_ref[both], axis=1)
                                                              / np.linalg.norm(z_ref[both], axis=1))),
               "max_rel_dJ_vs_projected_start": float(np.max(np.abs(Jf[both] - J_ref[both]) / J_ref[both]))}
        if s is not None:
            err = np.linalg.norm(s - z_ref, axis=1) / np.linalg.norm(z_ref, axis=1)
            row["median_start_err"] = float(np.median(err))
        if name == "mlp":
            mlp_status, mlp_z, mlp_J = stat, zf, Jf
        rows[name] = row
    out["starts"] = rows
    given.close()
    paper.close()

    # the plain FP64 one-query form on a sample of the same queries
    one = ift.Context.from_workload(wl, precision=ift.FP64, tol=1e-8, stream=stream.cuda_stream)
    one.set_eq_weights(rho_set)
    n1 = min(single_sample, n_query)
    one.solve_rom(mu_q[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    singles = [one.solve_rom(mu_q[q]) for q in range(n1)]
    dt = time.perf_counter() - t0
    # accuracy of the learned-start batched form against the FP64 one-query solves of
    # the same queries: both pass the same FP64 stopping test
    z1 = np.array([np.concatenate([r["w"], r["tau"]]) for r in singles])
    J1 = np.array([r["J"] for r in singles])
    ok1 = np.array([r["status"] == 0 for r in singles]) & (mlp_status[:n1] == 0)
    out["fp64_one_query"] = {
        "sample": n1, "solves_per_s": n1 / dt, "converged": int(sum(r["status"] == 0 for r in singles)),
        "mlp_batched_max_rel_dz": float(np.max(np.linalg.norm(mlp_z[:n1][ok1] - z1[ok1], axis=1)
                                               / np.linalg.norm(z1[ok1], axis=1))),
        "mlp_batched_max_rel_dJ": float(np.max(np.abs(mlp_J[:n1][ok1] - J1[ok1]) / J1[ok1]))}
    out["speedup_mlp_batched_vs_fp64_one_query"] = rows["mlp"]["solves_per_s"] / (n1 / dt)
    one.close()
    # Both forms meet the same stopping test, |[S; T]| <= 1e-8 max(1, |[S0; T0]|), and
    # here max(1, .) = 1 for every query: an absolute 1e-8. Their points still differ
    # where the hyperreduced problem is flat: the sample reports the final gradients,
    # the signed objective difference and the conditioning of the Gauss-Newton H at
    # the learned start's point (FP64 evaluation).
    one = ift.Context.from_workload(wl, precision=ift.FP64, tol=1e-8, stream=stream.cuda_stream)
    one.set_eq_weights(rho_set)
    g1s, g2s, dJs, lam_min, conds = [], [], [], [], []
    for q in range(n1):
        if not ok1[q]:
            continue
        ev = one.reduced_residual_jacobian(mu_q[q], mlp_z[q, :ku], mlp_z[q, ku:])
        lam = np.linalg.eigvalsh(ev["H"])
        g1s.append(float(np.linalg.norm(np.concatenate([ev["S"], ev["T"]]))))
        g2s.append(math.hypot(singles[q]["normS"], singles[q]["normT"]))
        dJs.append(float((mlp_J[q] - J1[q]) / J1[q]))
        lam_min.append(float(lam[0]))
        conds.append(float(lam[-1] / lam[0]))
    one.close()
    out["same_test_comparison"] = {
        "sample": len(dJs), "threshold": 1e-8,
        "max_final_gradient_mlp_batched": float(max(g1s)), "max_final_gradient_fp64_one_query": float(max(g2s)),
        "median_rel_dJ_mlp_minus_one_query": float(np.median(dJs)), "min_rel_dJ": float(min(dJs)),
        "max_rel_dJ": float(max(dJs)), "median_lambda_min_gn": float(np.median(lam_min)),
        "median_condition_number_gn": float(np.median(conds))}
    return out


def run_burgers(args):
    """Config 1: steady Burgers, p = 2, 200 elements, k_u = 5, k_x = 2, rho = 1, one
    ROM solve to a relative optimality of 1e-10 per step (a latency-bound solve:
    about 20 LM bodies over 200 elements)."""
    import torch

    import oracle as orc
    from paper_2305_15661_gb300 import ift
    from paper_2305_15661_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    ift.load()
    wl = W.burgers_workload(n_elems=200, p=2, k_u=5, seed=1)
    stream = torch.cuda.Stream(device=dev)
    ctx = ift.Context.from_workload(wl, tol=1e-10, stream=stream.cuda_stream)
    mu_d = torch.as_tensor(wl.mus[0], dtype=torch.float64, device=dev)
    y_d = torch.zeros(wl.ku, dtype=torch.float64, device=dev)
    z_d = torch.zeros(wl.kx, dtype=torch.float64, device=dev)
    info = None
    for _ in range(args.warmup):
        info = ctx.solve_rom_dev(mu_d, y_d, z_d, stream=stream.cuda_stream, want_info=True)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve_rom_dev(mu_d, y_d, z_d, stream=stream.cuda_stream, want_info=False)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    O = orc.Oracle.from_workload(wl)
    t0 = time.perf_counter()
    r = O.solve(wl.Phi, wl.Psi, wl.mus[0], wl.Phi.T @ W.replicate_guess(wl, wl.U_guess), tol=1e-10)
    cpu_s = time.perf_counter() - t0
    z = np.concatenate([y_d.cpu().numpy(), z_d.cpu().numpy()])
    zr = np.concatenate([r["w"], r["tau"]])
    print(json.dumps({"mode": "burgers", "elements": wl.n_elems, "p": wl.p, "k_u": wl.ku, "k_x": wl.kx,
                      "tol": 1e-10, "median_ms": statistics.median(ms), "solves_per_s": 1e3 / statistics.median(ms),
                      "lm_steps": info["init_iters"] + info["iters"], "oracle_lm_steps": r["init_iters"] + r["iters"],
                      "rel_dz_vs_oracle": float(np.linalg.norm(z - zr) / np.linalg.norm(zr)),
                      "cpu_oracle_s": cpu_s, "cpu_oracle_cores": orc.num_threads()}))
    ctx.close()
    return 0


def run_precisions(args):
    """Single-query ROM solves of the benchmark workload (20,000 elements, p = 2,
    k = 20 + 4, rho = 1, tol 1e-8) in each precision mode: FP64; FP32 Jacobians and
    contraction with the FP64 residual and gradient at every iteration; the
    two-stage mixed solve. Converged points compared with the FP64 solve."""
    import torch

    from paper_2305_15661_gb300 import ift

    dev = torch.device("cuda", 0)
    ift.load()
    wl = make_workload()
    stream = torch.cuda.Stream(device=dev)
    out = {"mode": "precisions", "workload": WORKLOAD, "tol": 1e-8, "solves": {}}
    ref = None
    for name, prec, contr in (("fp64", ift.FP64, ift.CONTRACT_FP), ("fp32jac", ift.FP32_JACOBIAN, ift.CONTRACT_FP),
                              ("fp32jac_tf32", ift.FP32_JACOBIAN, ift.CONTRACT_TF32),
                              ("mixed", ift.MIXED, ift.CONTRACT_FP)):
        ctx = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream, contraction=contr)
        ctx.autotune(wl.mus[0], wl.w_eval, wl.tau_eval)
        mu_d = torch.as_tensor(wl.mus[0], dtype=torch.float64, device=dev)
        y = torch.zeros(wl.ku, dtype=torch.float64, device=dev)
        z = torch.zeros(wl.kx, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            info = ctx.solve_rom_dev(mu_d, y, z, stream=stream.cuda_stream, want_info=True)
        ms = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.solve_rom_dev(mu_d, y, z, stream=stream.cuda_stream, want_info=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        zz = np.concatenate([y.cpu().numpy(), z.cpu().numpy()])
        row = {"ms": statistics.median(ms), "solves_per_s": 1e3 / statistics.median(ms), "status": info["status"],
               "lm_steps": info["init_iters"] + info["iters"] + info["fp32_iters"], "J": info["J"]}
        if ref is None:
            ref = zz
        else:
            row["rel_dz_vs_fp64"] = float(np.linalg.norm(zz - ref) / np.linalg.norm(ref))
        out["solves"][name] = row
        ctx.close()
    print(json.dumps(out))
    return 0


def run_greedy(args):
    """Greedy search (Eq. greedy0) over 256 candidate parameters on the 20,000-element
    mesh: batched hyperreduced solves with one shared weight set, then the full HDM
    residual norm (every element, no Jacobians) at each solution."""
    import torch

    from paper_2305_15661_gb300 import ift, perfmodel
    from paper_2305_15661_gb300 import workloads as W

    ift.load()
    B = args.candidates
    wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)
    rho = W.eq_weight_sets(wl, 1, seed=3, lo=400, hi=401)[0]
    mus = W.mu_box_samples(7, 1, B)
    prec = _precision(args)
    stream = torch.cuda.Stream(device=torch.device("cuda", 0))
    ctx = ift.Context.from_workload(wl, precision=prec, tol=1e-8, stream=stream.cuda_stream,
                                    contraction=_contraction(args))
    ctx.set_eq_weights_batched([rho] * B)
    shapes = ctx.autotune(mus[0], wl.w_eval, wl.tau_eval)
    res = ctx.solve_rom_batched(mus)
    ys, zs = res["w"], res["tau"]
    for _ in range(args.warmup):
        ctx.hdm_residual_norms(mus, ys, zs)
    ts, tn = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = ctx.solve_rom_batched(mus)
        t1 = time.perf_counter()
        norms = ctx.hdm_residual_norms(mus, res["w"], res["tau"])
        t2 = time.perf_counter()
        ts.append(t1 - t0)
        tn.append(t2 - t1)
    fl = perfmodel.flops_per_element(2, 2, wl.ku, wl.kx, jac=False)["total"]
    tnm = statistics.median(tn)
    print(json.dumps({"mode": "greedy", "precision": args.precision, "candidates": B, "elements": wl.n_elems,
                      "rho_nnz": int(len(rho[0])), "launch_shapes": shapes,
                      "solve_s": statistics.median(ts), "indicator_s": tnm,
                      "indicator_element_evals_per_s": B * wl.n_elems / tnm,
                      "indicator_tflops": B * wl.n_elems * fl / tnm / 1e12, "flops_per_element_residual": fl,
                      "argmax": int(np.argmax(norms)), "max_norm": float(np.max(norms)),
                      "median_norm": float(np.median(norms)),
                      "converged": int(sum(i["status"] == 0 for i in res["info"]))}))
    ctx.close()
    return 0


def run_align(args):
    """Snapshot alignment (Eq. align0) on the 20,000-element p = 2 mesh (--config 4:
    80,000 elements, p = 3, k_u = 40): a fixed
    number of full-space Levenberg-Marquardt steps on (w, interior mesh nodes) from
    the reference mesh, every element weighted 1. At each accepted point one element
    pass stores every element's block A_e = [dR_e/dw | dR_e/dx_e]; each
    conjugate-gradient iteration then reads those blocks once (J^T J v). The line
    reports wall time per alignment through the public call (host buffers in and
    out) and the device time of its phases (CUDA events inside the call)."""
    from paper_2305_15661_gb300 import ift
    from paper_2305_15661_gb300 import workloads as W

    ift.load()
    if args.config == 4:  # p = 3 on 200 x 200 x 2 triangles, k_u = 40
        wl = W.euler_workload(n=200, p=3, k_u=40, k_x=8, seed=4)
    else:
        wl = W.euler_workload(n=100, p=2, k_u=20, k_x=4, seed=2)
    ctx = ift.Context.from_workload(wl, kappa=0.1, align_cg_tol=args.align_cg_tol)
    mu = wl.mus[0]
    inner = np.all((wl.X > 1e-12) & (wl.X < 1 - 1e-12), axis=1)
    mask = np.repeat(inner, 2)
    x0 = wl.X.ravel()
    iters = args.align_iters
    for _ in range(args.warmup):
        ctx.align(mu, wl.w_eval, x0, mask, tol=0.0, max_iters=iters)
    ts, infos = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = ctx.align(mu, wl.w_eval, x0, mask, tol=0.0, max_iters=iters)
        ts.append(time.perf_counter() - t0)
        infos.append(r)
    t = statistics.median(ts)
    r = infos[len(infos) // 2]
    ne, nxe, nv = wl.n_elems, ctx.nxe, 3
    n = wl.ku + int(mask.sum())
    # one CG iteration: per element the coupling (M_e)_wx both ways and (M_e)_xx
    # (2 (2 k_u n_xe + n_xe^2) flops over k_u n_xe + n_xe^2 doubles, with the element's
    # direction and nodes), H_ww p_w once (2 k_u^2), plus about 14 passes over vectors
    # of the unknowns (product rows, dot, update, direction)
    blk = wl.ku * nxe + nxe * nxe
    cg_flops = 2.0 * ne * (2 * wl.ku * nxe + nxe * nxe) + 2.0 * wl.ku * wl.ku
    cg_bytes = ne * blk * 8 + ne * nxe * 8 + ne * nv * 4 + 14 * n * 8
    ms_cg_iter = r["ms_cg"] / max(r["cg_iters"], 1)
    fp64 = fp64_alu_peak()
    hbm = measured_peaks().get("hbm_gbs")
    tf = cg_flops / (ms_cg_iter * 1e-3) / 1e12
    gbs = cg_bytes / (ms_cg_iter * 1e-3) / 1e9
    print(json.dumps({"mode": "align", "elements": ne, "p": wl.p, "k_u": wl.ku, "free_coordinates": int(mask.sum()),
                      "cg_tol": args.align_cg_tol,
                      "lm_steps": r["iters"], "cg_iters": r["cg_iters"], "trials": r["trials"],
                      "s_per_alignment": t, "ms_form_per_point": r["ms_form"] / (r["iters"] + 1),
                      "ms_cg_per_iter": ms_cg_iter, "ms_search_per_trial": r["ms_search"] / max(r["trials"], 1),
                      "device_ms": {"form": r["ms_form"], "cg": r["ms_cg"], "search": r["ms_search"]},
                      "cg_iteration": {"flops": cg_flops, "bytes": cg_bytes, "fp64_tflops": tf,
                                       "fp64_peak": fp64, "frac_fp64": tf / fp64 if fp64 else None,
                                       "gbs": gbs, "hbm_peak": hbm, "frac_hbm": gbs / hbm if hbm else None,
                                       "note": "whole iteration (product and CG vector kernels); element "
                                               "systems %.0f MB (L2 129 MB)" % (ne * blk * 8 / 1e6)},
                      "J": r["J"], "gnorm_over_g0": r["gnorm"] / r["g0"], "status": r["status"]}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="default mode: skip the FP32-assembly, batched and warm-start keys")
    ap.add_argument("--mode", choices=["solve", "assembly", "batched", "warmstart", "greedy", "burgers", "precisions",
                                           "align"],
                    default="solve",
                    help="assembly: only time isolated fused assemblies (for profiler captures)")
    ap.add_argument("--precision", choices=["fp64", "fp32", "mixed", "fp32jac"], default="fp64",
                    help="element/contraction arithmetic for --mode assembly, batched and warmstart")
    ap.add_argument("--contraction", choices=["fp", "tf32", "3xtf32", "bf16"], default="fp",
                    help="FP32/mixed contexts: form H with FP32 FMAs, TF32 or 3xTF32 tensor cores")
    ap.add_argument("--config", type=int, choices=[2, 3, 4], default=2,
                    help="--mode assembly and align: 2 (or 3) = p 2, 20,000 elements, k 20+4; 4 = p 3, 80,000 "
                         "elements, k 40+8; --mode batched: 3 = 256 queries on the first mesh, 4 = 1,024 on the "
                         "second")
    ap.add_argument("--max-iters", type=int, default=200,
                    help="--mode batched: LM iterations per phase before a query stops unconverged")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="--mode batched: also solve the queries with FP64 assemblies and compare")
    ap.add_argument("--autotune", action="store_true", help="--mode assembly: tune the launch shape first")
    ap.add_argument("--q", type=int, choices=[1, 2], default=1,
                    help="--mode assembly: geometry degree (2: curved six-node triangles, the same sizes)")
    ap.add_argument("--train-solves", type=int, default=2048, help="--mode warmstart: training solves")
    ap.add_argument("--queries", type=int, default=4096, help="--mode warmstart: served queries")
    ap.add_argument("--candidates", type=int, default=256, help="--mode greedy: candidate parameters")
    ap.add_argument("--epochs", type=int, default=1500, help="--mode warmstart: training epochs")
    ap.add_argument("--single-sample", type=int, default=32, help="--mode warmstart: one-query FP64 solves timed")
    ap.add_argument("--align-iters", type=int, default=5, help="--mode align: Levenberg-Marquardt steps per alignment")
    ap.add_argument("--align-cg-tol", type=float, default=1e-12,
                    help="--mode align: relative residual of the CG solves (1e-12: exact steps)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "assembly":
        return run_assembly(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "warmstart":
        return run_warmstart(args)
    if args.mode == "greedy":
        return run_greedy(args)
    if args.mode == "burgers":
        return run_burgers(args)
    if args.mode == "precisions":
        return run_precisions(args)
    if args.mode == "align":
        return run_align(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

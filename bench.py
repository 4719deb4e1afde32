#!/usr/bin/env python
"""Throughput of the asymptotic parareal hot path on one GB300.

Headline workload (the largest single-GPU configuration, the precision-sweep
instance): 1D rotating shallow water, N = 1024 grid points, eps = 1e-4,
nu = 1e-4, T = 10 over 512 slices, fine ETDRK4 step dt = 1e-5 (1954 steps of
9.995e-6 per slice), M = 128 quadrature points, seeded synthetic initial
spectrum (|k| <= 32, scale e^{-k^2/256}).

One timed step = one complete parareal solve through the C ABI
(arp_set_initial + arp_parareal_solve with K_max = 5): the coarse predictor
and five iterations, each a fine sweep of all slices, V = F - G, the serial
chain of coarse steps and the convergence norm, pipelined across iterations
(ARP_OPT_PIPELINE).  Metric: fine grid-point-steps per second = 5 sweeps *
slices * N * fine steps / step time.  Beside it the line carries the same
solve on the single large instance (N = 512, 256 slices, M = 64), the time to
1e-5 relative error of the FP32-bulk solve against the plain FP64 GPU path,
serving latency (p50/p99) at one seeded Poisson rate, and the FP64 oracle on
the host cores, single-threaded and in parallel over slices.

--impl reference times the FP64 CPU oracle instead (one iteration restricted
to 2 slices per step, on the host cores).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rsw_inputs as ri  # noqa: E402

WORKLOAD = ri.SWEEP_N1024       # headline: the largest single-GPU configuration
LARGE = ri.LARGE_N512            # the single large instance, reported beside it
METRIC = "fine grid-pt-steps/s"
# FP32 peak of the plain ALUs: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz.
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64 peak: the part's nominal 1.25 TFLOP/s (FP64 units are a small fraction of FP32 ones).
FP64_ALU_PEAK_TFLOPS = 1.25
CPU_SAMPLE_SLICES = 8           # cpu_baseline sample, one core (about 10-20 s of oracle work at N = 1024)
CPU_PARALLEL_SLICES_PER_CORE = 2  # cpu_baseline sample in parallel over slices: slices per host core
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the fine-sweep kernel on a workload
# (ncu capture of the current kernel); None where no capture of the current kernel exists.
FINE_TRAFFIC_BYTES = {("rsw-N1024-eps1e-4-S512-M128", "fp32", 3): None,      # fine_sweep_kernel_f32_pairs<10,128>
                      ("rsw-N1024-eps1e-4-S512-M128", "fp32", 4): 8689408,   # fine_sweep_kernel_f32_r16<10,128>
                      ("rsw-N512-eps1e-3-S256-M64", "fp32", 2): 2256896}     # fine_sweep_kernel_f32<9,256>
REFERENCE_SAMPLE_SLICES = 2     # per-step sample of the reference arm


def flops_per_grid_pt_step(n_grid: int) -> float:
    """Algorithmic flops of one ETDRK4 step per grid point: 4 evaluations of N,
    each 7 real FFTs at 2.5 N log2 N, plus 52 N for rotations, derivatives and
    products; plus 80 N for the exponential combination."""
    return 70.0 * math.log2(n_grid) + 288.0


def solve_launches(slices: int, chunk: int, kmax: int) -> int:
    """Kernels one pipelined solve launches: per chunk of links the chain and
    the finish (at iterations with the per-slice change fused in), plus the
    correction at iterations, one max per iteration, and one fine launch per
    chunk with slices at levels 0 .. kmax-1."""
    n = -(-slices // chunk)
    fine = sum(1 for j in range(n)
               if min(slices, j * chunk + chunk + 1) > (0 if j == 0 else j * chunk + 1))
    return 2 * n + kmax * (3 * n + 1) + kmax * fine


def fine_steps(dT: float, dt: float) -> int:
    return max(1, int(math.ceil(dT / dt - 1e-9)))


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline solve (no N=512 solve, time to 1e-5 or serving keys)")
    ap.add_argument("--mode", choices=["headline", "tts", "precision", "batched", "serve", "paper", "schemes",
                                       "coarsegrid", "dftgemm", "kernels"],
                    default="headline",
                    help="headline: the contract line (default); tts: time to 1e-5 relative error against the "
                         "serial fine solution (FP64 sweeps on the GPU), FP32 bulk vs FP64; precision: the N=1024 precision sweep; "
                         "batched: 1024 uneven instances in one batch vs the FP64 path one instance at a time; "
                         "serve: Poisson request streams through the continuous-batching server; paper: the "
                         "experiments of Sec. 6.2 (Eq. 6.4 initial condition, eps = 1e-2, 1e-1, 1), asymptotic "
                         "and standard parareal; schemes: the three fine solvers' sweep throughput and "
                         "accuracy against the step size; coarsegrid: the coarse solver on N/2 and N/4 points; "
                         "dftgemm: the DFT-as-GEMM precisions against the FFT path; kernels: the predictor and "
                         "one level-by-level iteration of the headline workload (the whole-sweep fine launch and "
                         "the whole-chain cluster launch), a case for profilers")
    ap.add_argument("--instances", type=int, default=1024)
    ap.add_argument("--kernels-workload", choices=["n1024", "n512"], default="n1024",
                    help="with --mode kernels: the N=1024 headline workload or the N=512 instance")
    ap.add_argument("--fine-block", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="with --mode kernels: the FP32 fine sweep's schedule (ARP_OPT_FINE_BLOCK; 0 = tuned)")
    ap.add_argument("--probe", action="store_true",
                    help="with --mode dftgemm: only one small time average (a case sized for a profiler)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm

def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of the ranks' values (every rank gets it); the job's time is its
    slowest rank's.  Works with any initialised backend (NCCL with a CUDA device,
    gloo on the CPU)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank's replica does units_per_step per
    step, over the slowest rank's time."""
    return units_per_step * steps * world / (max_ms / 1e3)


def run_ours(args, rank: int, world: int, w=None, timed_steps: int | None = None) -> dict | None:
    """The contract line for workload w (default: the headline workload): complete
    solves timed on the device, the level-by-level solve beside them, the dominant
    kernel's own launch for the roofline, and the end-to-end solve with host buffers."""
    import torch
    import torch.distributed as dist

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(bld.LIB):
        bld.build()
    if world > 1:
        dist.barrier()
    b.load_library()
    w = w or WORKLOAD
    nsteps = timed_steps or args.steps
    steps = fine_steps(w.dT, w.dt)
    units = w.slices * w.n_grid * steps  # fine grid-point-steps per iteration
    prec = b.ARP_FP32 if args.precision == "fp32" else b.ARP_FP64
    H = w.n_grid // 2 + 1
    solver = b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec)
    ctx = solver.ctx
    stream = torch.cuda.current_stream()
    u0 = torch.from_numpy(w.initial_state()).cuda()
    kmax = w.k_max
    b.arp_set_option(ctx, b.ARP_OPT_KMAX, kmax)
    sweeps = kmax                                  # fine sweeps of one solve (levels 0 .. K_max-1)

    def solve():
        b.arp_set_initial(ctx, u0)
        return b.arp_parareal_solve(ctx)

    for _ in range(args.warmup):
        solve()
    # inputs are far smaller than L2 (129 MB): flush L2 between timed steps
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    changes = []
    for i in range(nsteps):
        flush.zero_()
        ev[i][0].record(stream)
        k_done, ch = solve()
        ev[i][1].record(stream)
        changes.append(ch)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    pinfo = b.arp_pipeline_info(ctx)
    step_ms = [a.elapsed_time(z) for a, z in ev]
    total_ms = max_over_ranks(sum(step_ms), world, "cuda")
    value = job_throughput(sweeps * units, nsteps, world, total_ms)
    launches = solve_launches(w.slices, pinfo["chunk"], kmax) if pinfo["pipelined"] else 5 * kmax + 2

    # the same solves level by level (no overlap of iterations), for comparison
    b.arp_set_option(ctx, b.ARP_OPT_PIPELINE, 0)
    solve()
    lbl = []
    for _ in range(min(nsteps, 5)):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solve()
        z.record(stream)
        lbl.append((a, z))
    torch.cuda.synchronize()
    lbl_ms = statistics.mean(a.elapsed_time(z) for a, z in lbl)
    b.arp_set_option(ctx, b.ARP_OPT_PIPELINE, 1)

    # dominant kernel: the fine sweep over all slices, timed live with events on its stream
    U = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
    b.arp_get_slices(ctx, U)
    Fin = U[:-1].contiguous()
    Fout = torch.empty_like(Fin)
    b.arp_fine_batch(ctx, Fin, Fout)
    reps = 5
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, z in fe:
        flush.zero_()
        a.record(stream)
        b.arp_fine_batch(ctx, Fin, Fout)
        z.record(stream)
    torch.cuda.synchronize()
    fine_ms = statistics.mean(a.elapsed_time(z) for a, z in fe)
    flops = units * flops_per_grid_pt_step(w.n_grid)
    achieved = flops / (fine_ms / 1e3) / 1e12
    peak = FP32_ALU_PEAK_TFLOPS if prec == b.ARP_FP32 else FP64_ALU_PEAK_TFLOPS
    peak_measured = b.arp_alu_peak(prec)  # FMA chains on every SM, this GPU
    sched = b.arp_info(ctx)["fine_schedule"]

    # end to end through the public API with host buffers: one complete solve per step
    # (u0 from pinned host memory, predictor + KMAX iterations, all slices back to pinned host)
    u0h = torch.from_numpy(w.initial_state()).pin_memory()
    Uh = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128).pin_memory()
    e2e_reps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        b.arp_set_initial(ctx, u0h)
        b.arp_parareal_solve(ctx)
        b.arp_get_slices(ctx, Uh)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_reps
    e2e_value = sweeps * units * world / e2e_s

    solver.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC,
        "value": value,
        "unit": "grid-pt-steps/s",
        "n_gpus": world,
        "steps": nsteps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / nsteps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == b.ARP_FP32 else "f64",
        "data": "synthetic (seeded spectra; no dataset in the paper)",
        "config": {"workload": w.name, "N": w.n_grid, "eps": w.eps, "nu": w.nu, "T": w.t_end,
                   "slices": w.slices, "dt": w.dt, "fine_steps_per_slice": steps, "M": w.m_quad,
                   "step": (f"one complete solve: coarse predictor + {kmax} parareal iterations (fine sweep, "
                            "correction, serial coarse chain, norm), pipelined across iterations"),
                   "pipeline": pinfo,
                   "precision": ("fp32 bulk, fp64 correction/norm/phases" if prec == b.ARP_FP32 else "fp64"),
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": FINE_TRAFFIC_BYTES.get((w.name, args.precision, sched)),
                     "kernel": ({3: "fine_sweep_kernel_f32_pairs", 4: "fine_sweep_kernel_f32_r16"}.get(
                                    sched, "fine_sweep_kernel_f32") if prec == b.ARP_FP32 else "fine_sweep_kernel"),
                     "fine_schedule": sched,
                     "launch_ms": fine_ms, "flop_per_launch": flops,
                     "peak_source": ("FP32 ALU: 152 SMs x 128 lanes x 2 x 2.07 GHz" if prec == b.ARP_FP32
                                     else "FP64 nominal 1.25 TFLOP/s"),
                     "peak_measured": peak_measured, "frac_of_measured": achieved / peak_measured,
                     "peak_measured_source": "arp_alu_peak: FMA register chains on every SM, timed with events"},
        "fine_only": {"value": units / (fine_ms / 1e3), "unit": "grid-pt-steps/s", "ms": fine_ms},
        "e2e": {"value": e2e_value, "unit": "grid-pt-steps/s", "h2d_bytes_per_step": int(u0h.numel() * 16),
                "d2h_bytes_per_step": int(Uh.numel() * 16),
                "step": f"complete solve: predictor + {kmax} iterations, host buffers", "seconds": e2e_s},
        "level_by_level": {"value": sweeps * units / (lbl_ms / 1e3), "unit": "grid-pt-steps/s",
                           "ms_per_step": lbl_ms, "note": "the same solves with ARP_OPT_PIPELINE 0"},
        "gpu_launches": nsteps * launches,
        "clocks": clk,
        "last_rel_change": changes[-1] if changes else None,
        "k_done": k_done,
    }


# ----------------------------------------------------------------------------- oracle on the host

def _oracle_params(w):
    from oracle import rsw as o
    return o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)


def oracle_predictor(slices: int, w=None):
    """The oracle's coarse predictor U^0 on the first `slices` slices of workload w."""
    import numpy as np

    from oracle import rsw as o
    w = w or WORKLOAD
    p = _oracle_params(w)
    U = [o.project(w.initial_state(), w.n_grid)]
    for _ in range(slices):
        U.append(o.coarse_step(U[-1], p))
    return np.stack(U)


def oracle_iteration_sample(slices: int, w=None, U=None):
    """One parareal iteration of the FP64 oracle on the first `slices` slices of
    workload w, starting from the predictor (computed untimed unless given);
    one host core.  Returns (seconds, fine grid-point-steps of the sample)."""
    from oracle import rsw as o
    w = w or WORKLOAD
    p = _oracle_params(w)
    U = oracle_predictor(slices, w) if U is None else U
    t0 = time.perf_counter()
    f_old = o.fine_propagate(U[:-1], p)
    g_old = o.coarse_step(U[:-1], p)
    new = [U[0]]
    for n in range(1, slices + 1):
        new.append(o.coarse_step(new[n - 1], p) + f_old[n - 1] - g_old[n - 1])
    dt = time.perf_counter() - t0
    return dt, slices * w.n_grid * fine_steps(w.dT, w.dt)


def _oracle_parallel_part(task):
    """Worker of the parallel oracle: F and G of one block of slices (the part
    of an iteration that is independent per slice)."""
    params, states = task
    from oracle import rsw as o
    p = o.Params(*params)
    return o.fine_propagate(states, p), o.coarse_step(states, p)


def _oracle_worker_ready(_):
    from oracle import rsw  # noqa: F401  (import cost paid before the timed region)
    return os.getpid()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_iteration_parallel(cores: int, per_core: int, w=None):
    """One parareal iteration of the FP64 oracle on cores x per_core slices of
    workload w, with F and G of the slices spread over `cores` worker processes
    (started with spawn, warmed up before the timed region) and the serial chain
    in this process.  Returns (seconds, units, slices)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import numpy as np

    from oracle import rsw as o
    w = w or WORKLOAD
    slices = cores * per_core
    p = _oracle_params(w)
    U = oracle_predictor(slices, w)
    params = (w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    # one numerical thread per worker: the cores are the workers
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_worker_ready, range(cores)))
            t0 = time.perf_counter()
            blocks = [U[i * per_core:(i + 1) * per_core] for i in range(cores)]
            parts = list(ex.map(_oracle_parallel_part, [(params, blk) for blk in blocks]))
            f_old = np.concatenate([f for f, _ in parts])
            g_old = np.concatenate([g for _, g in parts])
            new = [U[0]]
            for n in range(1, slices + 1):
                new.append(o.coarse_step(new[n - 1], p) + f_old[n - 1] - g_old[n - 1])
            dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return dt, slices * w.n_grid * fine_steps(w.dT, w.dt), slices


def cpu_cores_used() -> int:
    # numpy's FFT and the oracle's elementwise work are single-threaded
    return 1


def run_reference(args, rank: int) -> dict | None:
    if rank != 0:
        return None
    w = WORKLOAD
    times, units = [], 0
    U = oracle_predictor(REFERENCE_SAMPLE_SLICES, w)
    for i in range(args.warmup + args.steps):
        dt, units = oracle_iteration_sample(REFERENCE_SAMPLE_SLICES, w, U)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = units * args.steps / total
    sample = (f"one parareal iteration (fine sweep + G + serial chain) on {REFERENCE_SAMPLE_SLICES} of "
              f"{w.slices} slices per step")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "grid-pt-steps/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded spectra; no dataset in the paper)",
        "config": {"workload": w.name, "N": w.n_grid, "eps": w.eps, "nu": w.nu, "T": w.t_end,
                   "slices": w.slices, "dt": w.dt, "M": w.m_quad,
                   "step": sample},
        "cpu_baseline": {"value": value, "unit": "grid-pt-steps/s", "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "grid-pt-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------- other measurements

def _parseval(a):
    import numpy as np
    wgt = np.full(a.shape[-1], 2.0)
    wgt[0] = 1.0
    return np.sqrt(np.sum(wgt * np.abs(a) ** 2, axis=(-2, -1)))


def run_tts(args, w=None) -> dict:
    """Time to the first parareal iterate within 1e-5 (max over slices of the relative
    L2 error) of the serial fine solution, for the FP32-bulk and the plain FP64 path,
    one instance each, end to end through the C ABI with host buffers (u0 in;
    predictor and iterations; all slices out).  The serial fine solution comes from
    the FP64 fine sweep chained slice by slice on the GPU (held to the FP64 oracle
    within 1e-10 by the GPU tests); it is computed once, untimed."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = w or LARGE
    H = w.n_grid // 2 + 1
    t0 = time.perf_counter()
    ser = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
    ser[0] = torch.from_numpy(w.initial_state()).cuda()
    with b.Solver(w.n_grid, w.eps, w.nu, 1, w.dT, w.dt, w.m_quad) as s:
        for n in range(w.slices):
            b.arp_fine_batch(s.ctx, ser[n:n + 1], ser[n + 1:n + 2])
    ref = ser.cpu().numpy()
    t_ref = time.perf_counter() - t0
    out = {"mode": "tts", "workload": w.name, "target": 1e-5,
           "reference": "serial fine solution, FP64 sweeps chained slice by slice on the GPU",
           "reference_seconds": t_ref}
    u0h = torch.from_numpy(w.initial_state()).pin_memory()
    Uh = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128).pin_memory()
    kcap = 8
    for name, prec in (("fp64", b.ARP_FP64), ("fp32", b.ARP_FP32)):
        with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
            errs, kstar = [], None
            b.arp_set_initial(s.ctx, u0h)
            for k in range(kcap + 1):
                b.arp_parareal_iterate(s.ctx)
                b.arp_get_slices(s.ctx, Uh)
                e = float(np.max(_parseval(Uh.numpy()[1:] - ref[1:]) / _parseval(ref[1:])))
                errs.append(e)
                if e <= 1e-5 and kstar is None:
                    kstar = k
                    break
            # timed: the solve a user makes once K is known (pipelined where it applies)
            b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, kstar if kstar is not None else kcap)
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b.arp_set_initial(s.ctx, u0h)
                b.arp_parareal_solve(s.ctx)
                b.arp_get_slices(s.ctx, Uh)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            e = float(np.max(_parseval(Uh.numpy()[1:] - ref[1:]) / _parseval(ref[1:])))
            pinfo = b.arp_pipeline_info(s.ctx)
        out[name] = {"k_star": kstar, "errors_per_k": errs, "seconds": min(times), "solve_error": e,
                     "pipelined": bool(pinfo["pipelined"])}
    if out["fp64"]["k_star"] is not None and out["fp32"]["k_star"] is not None:
        out["speedup_fp32_vs_fp64"] = out["fp64"]["seconds"] / out["fp32"]["seconds"]
    return out


def eq51_speedup(slices, fine_steps_per_slice, iters, tau_f=1.0, tau_c=1.0):
    """Eq. 5.1's complexity model: serial fine cost over the cost of `iters`
    parareal iterations (each a parallel fine sweep and a serial coarse chain)
    plus the coarse predictor."""
    N, M = slices, fine_steps_per_slice
    return tau_f * N * M / (iters * (tau_f * M + tau_c * N + tau_c) + tau_c * N)


def _linf_rel(U, ref, n_grid):
    """max over slices of max_{x, field} |U - ref| / max_{x, field} |ref| (physical L-inf)."""
    import numpy as np
    d = np.fft.irfft(U * n_grid, n=n_grid, axis=-1)
    r = np.fft.irfft(ref * n_grid, n=n_grid, axis=-1)
    return float(np.max(np.max(np.abs(d - r), axis=(-2, -1)) / np.max(np.abs(r), axis=(-2, -1))))


def run_paper(args) -> dict:
    """Sec. 6.2's experiments on the GPU (FP64): the initial condition of Eq. 6.4,
    eps = 1e-2, 1e-1, 1 with the printed steps, window and nodes; the asymptotic
    method (ETDRK4 fine solver) and standard parareal with the Strang coarse step
    at the printed coarse steps; max relative L-inf error against the serial fine
    solution per iteration k = 0..5; Eq. 5.1's estimated speedup with equal step
    costs (the paper's assumption) and with the step costs measured here, and the
    measured ratio of serial fine time to the time of the predictor plus 5
    iterations."""
    import numpy as np
    import torch

    import rsw_inputs as ri
    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    kmax = 5

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def serial_fine(e, dT, slices, u0):
        """u(n dT), n = 0..slices, by one-state fine sweeps chained on the GPU; and the sweep time per step."""
        H = e.n_grid // 2 + 1
        out = torch.empty((slices + 1, 3, H), dtype=torch.complex128, device="cuda")
        out[0] = torch.from_numpy(u0).cuda()
        with b.Solver(e.n_grid, e.eps, e.nu, 1, dT, e.dt, e.m_quad) as s:
            b.arp_fine_batch(s.ctx, out[0:1], out[1:2])  # warm-up
            e0, e1 = events()
            e0.record()
            for n in range(slices):
                b.arp_fine_batch(s.ctx, out[n:n + 1], out[n + 1:n + 2])
            e1.record()
            torch.cuda.synchronize()
        steps = fine_steps(dT, e.dt)
        return out.cpu().numpy(), e0.elapsed_time(e1) / 1e3, steps

    def parareal(e, dT, slices, u0, coarse, window=None):
        H = e.n_grid // 2 + 1
        U = torch.empty((slices + 1, 3, H), dtype=torch.complex128, device="cuda")
        its, times = [], []
        with b.Solver(e.n_grid, e.eps, e.nu, slices, dT, e.dt, e.m_quad, T0=window) as s:
            b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_SCHEME, coarse)
            for rep in range(2):  # the first pass warms up, the second is timed
                b.arp_set_initial(s.ctx, torch.from_numpy(u0).cuda())
                its, times = [], []
                for _ in range(kmax + 1):
                    e0, e1 = events()
                    e0.record()
                    b.arp_parareal_iterate(s.ctx)
                    e1.record()
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1) / 1e3)
                    b.arp_get_slices(s.ctx, U)
                    its.append(U.cpu().numpy())
            # the same levels as one arp_parareal_solve (pipelined where it applies)
            b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, kmax)
            solve_s = []
            for rep in range(2):
                b.arp_set_initial(s.ctx, torch.from_numpy(u0).cuda())
                e0, e1 = events()
                e0.record()
                b.arp_parareal_solve(s.ctx)
                e1.record()
                torch.cuda.synchronize()
                solve_s.append(e0.elapsed_time(e1) / 1e3)
            b.arp_get_slices(s.ctx, U)
            same = bool(np.array_equal(U.cpu().numpy(), its[-1]))
            solve = {"seconds": solve_s[-1], "pipelined": bool(b.arp_pipeline_info(s.ctx)["pipelined"]),
                     "equals_iterates": same}
        return its, times, solve

    out = {"mode": "paper", "precision": "fp64", "fine": "ETDRK4", "experiments": []}
    for e in ri.PAPER_EXPERIMENTS:
        u0 = ri.paper_initial_state(e.n_grid)
        ref, t_serial, steps = serial_fine(e, e.dT, e.slices, u0)
        its, times, solve = parareal(e, e.dT, e.slices, u0, 0, e.window)
        errs = [_linf_rel(U[1:], ref[1:], e.n_grid) for U in its]
        tau_f = t_serial / (e.slices * steps)          # one fine step of one slice
        tau_c = times[0] / e.slices                     # one link of the predictor's chain
        row = {"name": e.name, "eps": e.eps, "dT": e.dT, "dt": e.dt, "window_fast_time": e.window,
               "M": e.m_quad, "slices": e.slices, "N": e.n_grid, "fine_steps_per_slice": steps,
               "asymptotic": {"errors_per_k": errs, "seconds_per_call": times,
                              "eq51_equal_costs": None, "eq51_measured_costs": None},
               "tau_f_us": tau_f * 1e6, "tau_c_us": tau_c * 1e6, "serial_fine_seconds": t_serial}
        row["asymptotic"]["eq51_equal_costs"] = eq51_speedup(e.slices, steps, kmax)
        row["asymptotic"]["eq51_measured_costs"] = eq51_speedup(e.slices, steps, kmax, tau_f, tau_c)
        row["asymptotic"]["measured_speedup"] = t_serial / sum(times)
        row["asymptotic"]["solve"] = dict(solve, measured_speedup=t_serial / solve["seconds"])
        row["standard"] = []
        for dT in e.standard_dT:
            S = int(round(e.t_end / dT))
            ref_s, t_ser_s, steps_s = serial_fine(e, dT, S, u0)
            its_s, times_s, _ = parareal(e, dT, S, u0, 1)
            errs_s = [_linf_rel(U[1:], ref_s[1:], e.n_grid) for U in its_s]
            tc_s = times_s[0] / S
            tf_s = t_ser_s / (S * steps_s)
            row["standard"].append({"dT": dT, "slices": S, "fine_steps_per_slice": steps_s, "errors_per_k": errs_s,
                                    "seconds_per_call": times_s, "tau_c_us": tc_s * 1e6,
                                    "eq51_equal_costs": eq51_speedup(S, steps_s, kmax),
                                    "eq51_measured_costs": eq51_speedup(S, steps_s, kmax, tf_s, tc_s),
                                    "measured_speedup": t_ser_s / sum(times_s)})
        out["experiments"].append(row)
        print(json.dumps({"done": e.name, "errors": errs}), file=sys.stderr, flush=True)
    return out


def scheme_flops_per_grid_pt_step(scheme: int, n_grid: int) -> float:
    """Algorithmic flops per grid-point-step of the fine schemes: ETDRK4 and
    integrating-factor RK4 evaluate N four times per step (flops_per_grid_pt_step),
    Strang splitting twice (2 x (17.5 log2 N + 52)) plus 20 for its combination."""
    if scheme == 1:
        return 35.0 * math.log2(n_grid) + 124.0
    return flops_per_grid_pt_step(n_grid)


def run_schemes(args) -> dict:
    """The three fine solvers (ETDRK4, Strang splitting, integrating-factor RK4):
    (1) one sweep of the large workload (256 slices, N = 512, 391 steps) per
    scheme and precision, with algorithmic throughput against the ALU peak;
    (2) accuracy at the step sizes Sec. 6.2 compares (dt = eps/10 .. eps/50 at
    eps = 1e-2, N = 128, the Eq. 6.4 initial condition, one coarse step of the
    experiment, dT = 0.5): max relative L-inf error against ETDRK4 at eps/400,
    all in FP64 on the GPU."""
    import numpy as np
    import torch

    import rsw_inputs as ri
    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = LARGE
    names = {0: "etdrk4", 1: "strang", 2: "ifrk4"}
    out = {"mode": "schemes", "workload": w.name, "sweep": {}, "accuracy": {}}
    x = torch.from_numpy(ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, w.slices, 9)).cuda()
    y = torch.empty_like(x)
    steps = fine_steps(w.dT, w.dt)
    for prec, pname, peak in ((b.ARP_FP32, "fp32", FP32_ALU_PEAK_TFLOPS), (b.ARP_FP64, "fp64", FP64_ALU_PEAK_TFLOPS)):
        for sch in (0, 1, 2):
            with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
                b.arp_set_option(s.ctx, b.ARP_OPT_FINE_SCHEME, sch)
                b.arp_fine_batch(s.ctx, x, y)
                torch.cuda.synchronize()
                ts = []
                for _ in range(5 if prec == b.ARP_FP32 else 2):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.arp_fine_batch(s.ctx, x, y)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            units = w.slices * w.n_grid * steps
            tf = units * scheme_flops_per_grid_pt_step(sch, w.n_grid) / (ms * 1e-3) / 1e12
            out["sweep"][f"{names[sch]}_{pname}"] = {"ms": ms, "grid_pt_steps_per_s": units / (ms * 1e-3),
                                                     "tflops": tf, "frac_of_alu_peak": tf / peak}
    # accuracy against the step size
    e = ri.PAPER_EXPERIMENTS[0]
    n, dT = e.n_grid, e.dT
    u0 = torch.from_numpy(ri.paper_initial_state(n)[None]).cuda()

    def sweep(scheme, dt):
        o_ = torch.empty_like(u0)
        with b.Solver(n, e.eps, e.nu, 1, dT, dt, e.m_quad) as s:
            b.arp_set_option(s.ctx, b.ARP_OPT_FINE_SCHEME, scheme)
            b.arp_fine_batch(s.ctx, u0, o_)
        return o_.cpu().numpy()

    ref = sweep(0, e.eps / 400)
    for sch in (0, 1, 2):
        row = {}
        for div in (10, 20, 25, 50):
            row[f"eps/{div}"] = _linf_rel(sweep(sch, e.eps / div), ref, n)
        out["accuracy"][names[sch]] = row
    return out


def run_coarsegrid(args) -> dict:
    """The asymptotic coarse solver on a coarser spatial grid (ARP_OPT_COARSE_GRID)
    at the large workload, FP32 bulk: for N_c = N, N/2, N/4, the time per parareal
    iteration and of its chain, and the max relative L2 error of the iterates
    k = 0..5 against the serial fine solution (FP64 sweeps chained on the GPU)."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = LARGE
    H = w.n_grid // 2 + 1
    u0 = torch.from_numpy(w.initial_state()).cuda()
    ser = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
    ser[0] = u0
    with b.Solver(w.n_grid, w.eps, w.nu, 1, w.dT, w.dt, w.m_quad) as s:
        for n in range(w.slices):
            b.arp_fine_batch(s.ctx, ser[n:n + 1], ser[n + 1:n + 2])
    ref = ser.cpu().numpy()
    out = {"mode": "coarsegrid", "workload": w.name, "precision": "fp32", "runs": []}
    U = torch.empty_like(ser)
    for nc in (w.n_grid, w.n_grid // 2, w.n_grid // 4):
        with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=b.ARP_FP32) as s:
            b.arp_set_option(s.ctx, b.ARP_OPT_COARSE_GRID, nc)
            errs, ms = [], []
            for rep in range(2):  # the first pass warms up (and creates the coarse sub-context)
                b.arp_set_initial(s.ctx, u0)
                errs, ms = [], []
                for k in range(6):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.arp_parareal_iterate(s.ctx)
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    b.arp_get_slices(s.ctx, U)
                    x = U.cpu().numpy()
                    errs.append(float(np.max(_parseval(x[1:] - ref[1:]) / _parseval(ref[1:]))))
        out["runs"].append({"N_c": nc, "errors_per_k": errs, "predictor_ms": ms[0],
                            "ms_per_iteration": statistics.median(ms[1:])})
    return out


def run_dftgemm(args) -> dict:
    """The DFT-as-GEMM precisions against the FFT path on the large workload:
    one fine sweep of the 256 slices (391 ETDRK4 steps, all slices stepped
    together in the GEMM precisions) and one batched time average of the 256
    states over M = 64 nodes; wall time per call, algorithmic TFLOP/s counted
    with FFT flops (so the dense 2 N (2K+1) flops per transform get no credit),
    and the rate of the dense GEMM work itself."""
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = LARGE
    if args.probe:
        # one time average per split precision on 64 states (4096 column groups), twice: a small case for a profiler
        x = torch.from_numpy(ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 64, 9)).cuda()
        y = torch.empty_like(x)
        for prec in (b.ARP_TF32X3, b.ARP_BF16X3):
            with b.Solver(w.n_grid, w.eps, w.nu, 64, w.dT, w.dt, w.m_quad, precision=prec) as s:
                for _ in range(2):
                    b.arp_coarse_avg(s.ctx, x, y)
        torch.cuda.synchronize()
        return {"mode": "dftgemm", "probe": "one ARP_TF32X3 and one ARP_BF16X3 time average of 64 states, twice each"}
    x = torch.from_numpy(ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, w.slices, 9)).cuda()
    y = torch.empty_like(x)
    steps = fine_steps(w.dT, w.dt)
    N, K = w.n_grid, (w.n_grid - 1) // 3
    R = 2 * K + 1
    out = {"mode": "dftgemm", "workload": w.name, "fine_sweep": {}, "time_average": {}}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    products = {b.ARP_TF32X3: 3, b.ARP_BF16X2: 4, b.ARP_BF16X3: 6}
    for name, prec in (("fp32_fft", b.ARP_FP32), ("tf32x3_gemm", b.ARP_TF32X3), ("bf16x2_gemm", b.ARP_BF16X2),
                       ("bf16x3_gemm", b.ARP_BF16X3)):
        with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
            ms = timed(lambda: b.arp_fine_batch(s.ctx, x, y), 3)
            units = w.slices * N * steps
            # dense work per step: 4 evaluations x (4 inverse + 3 forward columns) x 2 N R flops x split products
            dense = w.slices * steps * 4 * 7 * 2 * N * R * products.get(prec, 0)
            out["fine_sweep"][name] = {"ms": ms, "algorithmic_tflops": units * flops_per_grid_pt_step(N) / ms / 1e9,
                                       "dense_gemm_tflops": dense / ms / 1e9 if prec != b.ARP_FP32 else None}
            ms = timed(lambda: b.arp_coarse_avg(s.ctx, x, y), 5)
            nodes = w.slices * w.m_quad
            fft_flops = nodes * N * (35.0 * math.log2(N) + 64.0)  # one N-evaluation per node
            dense = nodes * 7 * 2 * N * R * products.get(prec, 0)
            out["time_average"][name] = {"ms": ms, "algorithmic_tflops": fft_flops / ms / 1e9,
                                         "dense_gemm_tflops": dense / ms / 1e9 if prec != b.ARP_FP32 else None}
    return out


def run_precision(args) -> dict:
    """Precision sweep on the N=1024 instance (eps=1e-4, 512 slices, 1954 fine steps,
    M=128): per-field relative L2 error of one fine sweep in FP32 bulk, 3xTF32 and
    2xBF16 DFT-GEMMs against the FP64 path (which the GPU tests hold to the FP64
    oracle within 1e-10) and the mean-height drift of each; then full-size parareal,
    FP32 against FP64 (iterates k = 0..3) and the time per iteration of each, and the
    FP32 solve of the same levels level by level and pipelined."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = ri.SWEEP_N1024
    H = w.n_grid // 2 + 1
    x = ri.random_batch(w.n_grid, w.ic_cutoff, w.ic_scale_div, 3, 500) * 64.0
    ref = None
    out = {"mode": "precision", "workload": w.name, "fine_sweep_vs_fp64": {}, "parareal_fp32_vs_fp64": {}}
    fields = ("v1", "v2", "h")
    iterates = {}
    for name, prec in (("fp64", b.ARP_FP64), ("fp32", b.ARP_FP32), ("tf32x3", b.ARP_TF32X3),
                       ("bf16x2", b.ARP_BF16X2), ("bf16x3", b.ARP_BF16X3)):
        with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
            xin = torch.from_numpy(x).cuda()
            y = torch.empty_like(xin)
            b.arp_fine_batch(s.ctx, xin, y)
            got = y.cpu().numpy()
            if ref is None:
                ref = got  # the FP64 sweep (first in this loop)
            rel = {f: float(np.max(np.linalg.norm(got[:, i] - ref[:, i], axis=-1) / np.linalg.norm(ref[:, i], axis=-1)))
                   for i, f in enumerate(fields)}
            drift = float(np.max(np.abs(got[:, 2, 0] - x[:, 2, 0].real) / np.abs(x[:, 2, 0].real)))
            out["fine_sweep_vs_fp64"][name] = {"rel_l2": rel, "mean_height_drift": drift}
            if prec in (b.ARP_TF32X3, b.ARP_BF16X2, b.ARP_BF16X3):
                continue  # the full-size parareal comparison below is FP32 against FP64
            b.arp_set_initial(s.ctx, torch.from_numpy(w.initial_state()).cuda())
            U = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
            its, ms = [], []
            for k in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b.arp_parareal_iterate(s.ctx)
                torch.cuda.synchronize()
                ms.append(1e3 * (time.perf_counter() - t0))
                b.arp_get_slices(s.ctx, U)
                its.append(U.cpu().numpy())
            iterates[name] = its
            out["parareal_fp32_vs_fp64"][name + "_ms_per_iteration"] = ms[1:]
            if prec == b.ARP_FP32:
                # the same three iterations as one solve, level by level and pipelined
                b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, 3)
                solve = {}
                for label, pipe in (("level_by_level", 0), ("pipelined", 1)):
                    b.arp_set_option(s.ctx, b.ARP_OPT_PIPELINE, pipe)
                    b.arp_set_initial(s.ctx, torch.from_numpy(w.initial_state()).cuda())
                    b.arp_parareal_solve(s.ctx)  # warm-up
                    ts = []
                    for _ in range(2):
                        b.arp_set_initial(s.ctx, torch.from_numpy(w.initial_state()).cuda())
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        b.arp_parareal_solve(s.ctx)
                        torch.cuda.synchronize()
                        ts.append(1e3 * (time.perf_counter() - t0))
                    solve[label + "_ms"] = min(ts)
                    solve[label + "_ran_pipelined"] = bool(b.arp_pipeline_info(s.ctx)["pipelined"])
                    b.arp_get_slices(s.ctx, U)
                    solve[label + "_equals_iterates"] = bool(np.array_equal(U.cpu().numpy(), its[3]))
                out["parareal_fp32_vs_fp64"]["fp32_solve_predictor_plus_3"] = solve
    d = []
    for k in range(4):
        a, r = iterates["fp32"][k][1:], iterates["fp64"][k][1:]
        d.append(float(np.max(_parseval(a - r) / _parseval(r))))
    out["parareal_fp32_vs_fp64"]["max_rel_l2_per_k"] = d
    h0 = w.initial_state()[2, 0].real
    out["parareal_fp32_vs_fp64"]["mean_height_drift_fp32"] = float(
        np.max(np.abs(iterates["fp32"][3][:, 2, 0].real - h0)) / abs(h0))
    return out


def run_batched(args) -> dict:
    """Batched uneven instances: `--instances` independent problems (N from
    {64..1024}, eps log-uniform in [1e-4, 1e-2], 32/64/128 slices, M = 32, T = 1,
    dt = eps/10) advanced together by arp_batch_iterate in FP32 bulk (predictor +
    5 iterations), against the plain FP64 path run one instance at a time on a
    seeded sample of 16 of them."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    insts = ri.uneven_instances(args.instances)
    units = [w.slices * w.n_grid * fine_steps(w.dT, w.dt) for w in insts]
    t0 = time.perf_counter()
    solvers = [b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=b.ARP_FP32) for w in insts]
    for s, w in zip(solvers, insts):
        b.arp_set_initial(s.ctx, torch.from_numpy(w.initial_state()).cuda())
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    batch = b.arp_batch_create([s.ctx for s in solvers])
    levels = 6
    ms = []
    for k in range(levels):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lv, ch = b.arp_batch_iterate(batch, len(solvers))
        ms.append(1e3 * (time.perf_counter() - t0))
    iter_ms = ms[1:]
    value = sum(units) / (statistics.mean(iter_ms) / 1e3)
    # sample: the plain FP64 path, one instance at a time
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(len(insts), size=min(16, len(insts)), replace=False).tolist())
    t_single, dev = 0.0, 0.0
    for i in sample:
        w = insts[i]
        H = w.n_grid // 2 + 1
        with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.arp_set_initial(s.ctx, torch.from_numpy(w.initial_state()).cuda())
            for _ in range(levels):
                b.arp_parareal_iterate(s.ctx)
            torch.cuda.synchronize()
            t_single += time.perf_counter() - t0
            U64 = torch.empty((w.slices + 1, 3, H), dtype=torch.complex128, device="cuda")
            b.arp_get_slices(s.ctx, U64)
        U32 = torch.empty_like(U64)
        b.arp_get_slices(solvers[i].ctx, U32)
        a, r = U32.cpu().numpy()[1:], U64.cpu().numpy()[1:]
        dev = max(dev, float(np.max(_parseval(a - r) / _parseval(r))))
    b.arp_batch_destroy(batch)
    for s in solvers:
        s.close()
    batch_total_s = sum(ms) / 1e3
    return {"mode": "batched", "instances": len(insts), "precision": "fp32 bulk, fp64 correction/norm/phases",
            "value": value, "unit": "fine grid-pt-steps/s", "ms_per_batched_iteration": iter_ms,
            "predictor_ms": ms[0], "setup_seconds": t_setup, "levels": levels,
            "batched_seconds_all_levels": batch_total_s,
            "fp64_single_sample": {"instances": len(sample), "seconds_all_levels": t_single,
                                   "extrapolated_seconds_all_instances": t_single * len(insts) / len(sample)},
            "speedup_vs_fp64_one_at_a_time": (t_single * len(insts) / len(sample)) / batch_total_s,
            "max_rel_l2_fp32_batched_vs_fp64_single": dev,
            "final_max_change": float(np.nanmax(np.array(ch)))}


def serve_requests(count: int, seed: int):
    """Seeded serving requests: N from {128..2048}, eps log-uniform in [1e-4, 1e-2],
    slices from {32..512}, T from {0.1, 0.5, 1}, dt = min(eps/10, T/slices), M = 32, at most 5
    iterations or a change <= 1e-8; initial spectra as the small workload's (|k| <= 8,
    scale e^{-k^2/16}), request i seeded seed + i."""
    from paper_1303_6615_gb300 import serve
    g = ri.SplitMix64(seed ^ 0x5E7E)
    out = []
    for i in range(count):
        n = (128, 256, 512, 1024, 2048)[g.next_u64() % 5]
        eps = 10.0 ** (-4.0 + 2.0 * g.uniform())
        S = (32, 64, 128, 256, 512)[g.next_u64() % 5]
        T = (0.1, 0.5, 1.0)[g.next_u64() % 3]
        u0 = ri.random_spectrum(n, 8, 16.0, seed + i)
        out.append(serve.Request(n, eps, 1e-4, S, T, min(eps / 10.0, T / S), 32, u0, k_max=5, tol=1e-8))
    return out


def run_serve(args) -> dict:
    """Poisson request streams (rates 10, 100, 1000 per second, 64 requests each)
    through the continuous-batching FP32 server (with and without the one-call
    solve of a request that runs alone), against the plain FP64 path
    serving the same requests one at a time in arrival order (first come first
    served, each request's FP64 service time measured on its own)."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    from paper_1303_6615_gb300 import serve
    bld.build()
    count = 64
    base = serve_requests(count, 3000)
    service64 = []
    for r in base:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        serve.solve_alone(r, b.ARP_FP64)
        torch.cuda.synchronize()
        service64.append(time.perf_counter() - t0)
    out = {"mode": "serve", "requests_per_rate": count, "fp64_one_at_a_time_service_s_mean": float(np.mean(service64)),
           "rates": {}}
    for rate in (10.0, 100.0, 1000.0):
        rng = np.random.default_rng(int(rate))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
        stats = {}
        for lone in (True, False):
            reqs = serve_requests(count, 3000)
            server = serve.Server(memory_budget=24 << 30, max_active=256, precision=b.ARP_FP32, lone_solve=lone)
            try:
                t0 = server.clock()
                done = serve.replay(server, list(zip(arrivals.tolist(), reqs)))
                makespan = server.clock() - t0
            finally:
                server.close()
            lat = np.array([r.latency for r in done])
            stats[lone] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                           "throughput_req_s": count / makespan}
        # first come first served, one at a time, FP64
        finish, lat64 = 0.0, []
        for a, s in zip(arrivals, service64):
            finish = max(finish, a) + s
            lat64.append(finish - a)
        lat64 = np.array(lat64)
        out["rates"][str(int(rate))] = {
            "batched_fp32": stats[True],
            "batched_fp32_levels_only": stats[False],
            "fp64_one_at_a_time": {"p50_s": float(np.percentile(lat64, 50)), "p99_s": float(np.percentile(lat64, 99)),
                                   "throughput_req_s": count / (finish - 0.0)},
        }
    return out


def serve_one_rate(rate: float = 100.0, count: int = 64, seed: int = 3000) -> dict:
    """Serving latency at one seeded Poisson rate: `count` requests (serve_requests)
    through the continuous-batching FP32 server, and the plain FP64 path serving
    the same requests one at a time in arrival order (each request's FP64 service
    time measured alone on the GPU)."""
    import numpy as np
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import serve
    rng = np.random.default_rng(int(rate))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = serve_requests(count, seed)
    server = serve.Server(memory_budget=24 << 30, max_active=256, precision=b.ARP_FP32, lone_solve=True)
    try:
        t0 = server.clock()
        done = serve.replay(server, list(zip(arrivals.tolist(), reqs)))
        makespan = server.clock() - t0
    finally:
        server.close()
    lat = np.array([r.latency for r in done])
    service64 = []
    for r in serve_requests(count, seed):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        serve.solve_alone(r, b.ARP_FP64)
        torch.cuda.synchronize()
        service64.append(time.perf_counter() - t1)
    finish, lat64 = 0.0, []
    for a, sv in zip(arrivals, service64):
        finish = max(finish, a) + sv
        lat64.append(finish - a)
    lat64 = np.array(lat64)
    return {"rate_req_s": rate, "requests": count, "seed": seed,
            "requests_mix": "N 128-2048, eps 1e-4-1e-2, 32-512 slices, T 0.1-1, M 32, K_max 5 or change <= 1e-8",
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "throughput_req_s": count / makespan,
            "fp64_one_at_a_time": {"p50_ms": 1e3 * float(np.percentile(lat64, 50)),
                                   "p99_ms": 1e3 * float(np.percentile(lat64, 99)),
                                   "throughput_req_s": count / finish}}


def run_kernels(args) -> dict:
    """A workload's two dominant kernels in their level-by-level launches
    (ARP_OPT_PIPELINE 0): the predictor's chain (one cluster launch over all
    links), then one iteration: the fine sweep of all slices in one launch, the
    correction, the chain, the norm.  --kernels-workload picks the headline
    workload (n1024, default) or the single large instance (n512)."""
    import torch

    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    w = WORKLOAD if args.kernels_workload == "n1024" else LARGE
    prec = b.ARP_FP32 if args.precision == "fp32" else b.ARP_FP64
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with b.Solver(w.n_grid, w.eps, w.nu, w.slices, w.dT, w.dt, w.m_quad, precision=prec) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_PIPELINE, 0)
        b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, args.fine_block)
        u0 = torch.from_numpy(w.initial_state()).cuda()
        for timed in (False, True):
            b.arp_set_initial(s.ctx, u0)
            if not timed:
                b.arp_parareal_iterate(s.ctx)
                b.arp_parareal_iterate(s.ctx)
        torch.cuda.synchronize()
        ev[0].record()
        b.arp_parareal_iterate(s.ctx)
        ev[1].record()
        k, ch = b.arp_parareal_iterate(s.ctx)
        ev[2].record()
        torch.cuda.synchronize()
        sched = b.arp_info(s.ctx)["fine_schedule"]
    return {"mode": "kernels", "workload": w.name, "precision": args.precision, "fine_schedule": sched,
            "level": k, "change": ch,
            "predictor_ms": ev[0].elapsed_time(ev[1]), "iteration_ms": ev[1].elapsed_time(ev[2]),
            "note": "one timed pass after one warm-up pass; a case for profilers, not the benchmark"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.mode != "headline":
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            res = {"tts": run_tts, "precision": run_precision, "batched": run_batched, "serve": run_serve,
                   "paper": run_paper, "schemes": run_schemes, "coarsegrid": run_coarsegrid,
                   "dftgemm": run_dftgemm, "kernels": run_kernels}[args.mode](args)
            print(json.dumps(res), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if out is not None:
        if world == 1 and not args.headline_only:
            # the same solve on the single large instance, the time to 1e-5 and serving latency
            big = run_ours(args, rank, world, LARGE, timed_steps=args.steps)
            out["config_N512"] = {k: big[k] for k in ("value", "unit", "ms_per_step", "config", "roofline", "e2e",
                                                      "level_by_level", "fine_only", "clocks")}
            tts = run_tts(args, LARGE)
            out["tts"] = {"workload": tts["workload"], "target_rel_l2": tts["target"],
                          "reference": tts["reference"],
                          "fp32_bulk_solve_s": tts["fp32"]["seconds"], "fp32_k": tts["fp32"]["k_star"],
                          "fp32_pipelined": tts["fp32"]["pipelined"], "fp32_error": tts["fp32"]["solve_error"],
                          "fp64_plain_solve_s": tts["fp64"]["seconds"], "fp64_k": tts["fp64"]["k_star"],
                          "fp64_error": tts["fp64"]["solve_error"],
                          "speedup_fp32_vs_fp64": tts.get("speedup_fp32_vs_fp64"),
                          "note": "end to end through the C ABI with host buffers, one instance each"}
            out["serve"] = serve_one_rate()
        if world == 1 and not args.no_cpu_baseline:
            U = oracle_predictor(CPU_SAMPLE_SLICES)
            dt, units = oracle_iteration_sample(CPU_SAMPLE_SLICES, WORKLOAD, U)
            cores = host_cores()
            dtp, unitsp, slp = oracle_iteration_parallel(cores, CPU_PARALLEL_SLICES_PER_CORE)
            out["cpu_baseline"] = {"value": units / dt, "unit": "grid-pt-steps/s", "cores": cpu_cores_used(),
                                   "kind": "oracle", "cpu": cpu_model(),
                                   "sample": f"one FP64 oracle parareal iteration on {CPU_SAMPLE_SLICES} of "
                                             f"{WORKLOAD.slices} slices ({dt:.1f} s), one core",
                                   "parallel": {"value": unitsp / dtp, "unit": "grid-pt-steps/s", "cores": cores,
                                                "sample": f"one FP64 oracle parareal iteration on {slp} of "
                                                          f"{WORKLOAD.slices} slices ({dtp:.1f} s), F and G of "
                                                          f"the slices in {cores} worker processes, the serial "
                                                          "chain in one"}}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

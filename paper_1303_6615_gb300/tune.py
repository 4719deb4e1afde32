"""Offline tuner of the FP32 fine sweep's schedule per grid size.

For every grid size N = 8 .. 2048 it times each schedule of the FP32 ETDRK4
fine sweep (ARP_OPT_FINE_BLOCK 1 = N/4 threads per slice, 2 = N/2 threads,
3 = N/8 threads with both FFT lanes per butterfly and the stage values in
shared memory, where it applies) on one GPU, through the C ABI, and writes
the fastest into csrc/fine_schedule.h together with every measured time.  The
library is then rebuilt with that table as its default.

The schedules round differently in the last bits, so the choice is made here,
offline, and stored: a run of the library never picks a schedule by timing,
and its results do not depend on timing noise.

Usage (on the GPU): python -m paper_1303_6615_gb300.tune [--slices 512] [--steps 64]
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HEADER = os.path.join(PKG, "csrc", "fine_schedule.h")
SCHEDULES = {1: "N/4 threads", 2: "N/2 threads", 3: "N/8 threads, lane pairs, shared stage values"}


def schedules_for(logn: int) -> list[int]:
    n = 1 << logn
    out = [1]
    if min(max(n // 2, 32), 512) != min(max(n // 4, 32), 512):
        out.append(2)
    if logn >= 8:
        out.append(3)
    return out


def time_schedule(b, torch, ri, n: int, slices: int, steps: int, sched: int, reps: int = 3) -> float:
    eps, dT = 1e-3, 1e-3 * steps / 10.0
    x = torch.from_numpy(ri.random_batch(n, min(32, (n - 1) // 3), 256.0, slices, 77)).cuda()
    y = torch.empty_like(x)
    with b.Solver(n, eps, 1e-4, slices, dT, dT / steps, 8, precision=b.ARP_FP32) as s:
        b.arp_set_option(s.ctx, b.ARP_OPT_FINE_BLOCK, sched)
        b.arp_fine_batch(s.ctx, x, y)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.arp_fine_batch(s.ctx, x, y)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def write_header(table: list[int], times: dict, slices: int, steps: int, gpu: str) -> None:
    lines = [
        "// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.",
        "// Default schedule of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):",
        "// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs.",
        f"// Measured on {gpu}: one sweep of {slices} slices x {steps} steps, median of 3, ms:",
    ]
    for logn in sorted(times):
        row = ", ".join(f"{k}: {v:.3f}" for k, v in sorted(times[logn].items()))
        lines.append(f"//   N = {1 << logn:5d}  {row}  -> {table[logn]}")
    lines += ["#pragma once", "", "namespace arp {", "",
              "constexpr int kFineScheduleF32[12] = {" + ", ".join(str(v) for v in table) + "};", "",
              "}  // namespace arp", ""]
    with open(HEADER, "w") as f:
        f.write("\n".join(lines))


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--slices", type=int, default=512)
    ap.add_argument("--steps", type=int, default=64)
    args = ap.parse_args()
    import torch

    import rsw_inputs as ri
    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    torch.cuda.set_device(0)
    table = [1] * 12
    times: dict[int, dict[int, float]] = {}
    for logn in range(3, 12):
        n = 1 << logn
        times[logn] = {s: time_schedule(b, torch, ri, n, args.slices, args.steps, s) for s in schedules_for(logn)}
        table[logn] = min(times[logn], key=times[logn].get)
        print(f"N={n}: " + ", ".join(f"{SCHEDULES[k]} {v:.3f} ms" for k, v in times[logn].items())
              + f" -> {table[logn]}", flush=True)
    write_header(table, times, args.slices, args.steps, torch.cuda.get_device_name(0))
    print(f"wrote {HEADER}")


if __name__ == "__main__":
    main()

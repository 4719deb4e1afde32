"""Offline tuner of the FP32 fine sweep's schedule per grid size.

For every grid size N = 8 .. 2048 it times each schedule of the FP32 ETDRK4
fine sweep (ARP_OPT_FINE_BLOCK 1 = N/4 threads per slice, 2 = N/2 threads,
3 = N/8 threads with both FFT lanes per butterfly and the stage values in
shared memory, 4 = N/8 threads with radix-16 transform stages and the stage
values in shared memory, where they apply) on one GPU, through the C ABI, in the two
regimes the library launches it in: a whole sweep of many slices (--slices,
several per SM: throughput, as a level-by-level iteration or a batch runs it)
and a chunk of a few slices (--chunk, well under one per SM: the per-slice
latency that bounds the pipelined solve, whose fine launches are chunks of the
chain's links).  It writes the fastest schedule of each regime into
csrc/fine_schedule.h (a throughput and a latency table) together with every
measured time, and the library is rebuilt with them: a context whose slices
fill the device (two or more per SM) takes the throughput table's schedule,
others the latency table's, for every launch (the pipelined and the
level-by-level solve of one context must run the same schedule to give the
same bits).

The schedules round differently in the last bits, so the choice is made here,
offline, and stored: a run of the library never picks a schedule by timing,
and its results do not depend on timing noise.

Usage (on the GPU): python -m paper_1303_6615_gb300.tune [--slices 512] [--chunk 16] [--steps 64]
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
SCHEDULES = {1: "N/4 threads", 2: "N/2 threads", 3: "N/8 threads, lane pairs, shared stage values",
             4: "N/8 threads, radix-16 stages, shared stage values"}


def schedules_for(logn: int) -> list[int]:
    n = 1 << logn
    out = [1]
    if min(max(n // 2, 32), 512) != min(max(n // 4, 32), 512):
        out.append(2)
    if logn >= 8:
        out.append(3)
    if 9 <= logn <= 11:
        out.append(4)
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


def pick(times: dict) -> int:
    """The fastest schedule of one regime."""
    return min(times, key=times.get)


def write_header(tp_table: list[int], lat_table: list[int], times: dict, lat: dict, slices: int, chunk: int,
                 steps: int, gpu: str) -> None:
    lines = [
        "// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.",
        "// Default schedules of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):",
        "// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs,",
        "// 4 = N/8 threads with radix-16 stages.",
        f"// Measured on {gpu}, {steps} steps, median of 3, ms: a sweep of {slices} slices (throughput)",
        f"// / of {chunk} slices (latency); the fastest of each regime is kept.",
    ]
    for logn in sorted(times):
        row = ", ".join(f"{k}: {times[logn][k]:.3f} / {lat[logn][k]:.3f}" for k in sorted(times[logn]))
        lines.append(f"//   N = {1 << logn:5d}  {row}  -> {tp_table[logn]} / {lat_table[logn]}")
    lines += ["#pragma once", "", "namespace arp {", "",
              "// contexts whose slices fill the device (at least two per SM)",
              "constexpr int kFineScheduleF32Tp[12] = {" + ", ".join(str(v) for v in tp_table) + "};",
              "// contexts with fewer slices",
              "constexpr int kFineScheduleF32Lat[12] = {" + ", ".join(str(v) for v in lat_table) + "};", "",
              "}  // namespace arp", ""]
    with open(HEADER, "w") as f:
        f.write("\n".join(lines))


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--slices", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=16)
    ap.add_argument("--steps", type=int, default=64)
    args = ap.parse_args()
    import torch

    import rsw_inputs as ri
    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import build as bld
    bld.build()
    torch.cuda.set_device(0)
    tp_table, lat_table = [1] * 12, [1] * 12
    times: dict[int, dict[int, float]] = {}
    lat: dict[int, dict[int, float]] = {}
    for logn in range(3, 12):
        n = 1 << logn
        times[logn] = {s: time_schedule(b, torch, ri, n, args.slices, args.steps, s) for s in schedules_for(logn)}
        lat[logn] = {s: time_schedule(b, torch, ri, n, args.chunk, args.steps, s) for s in schedules_for(logn)}
        tp_table[logn], lat_table[logn] = pick(times[logn]), pick(lat[logn])
        print(f"N={n}: " + ", ".join(f"{SCHEDULES[k]} {times[logn][k]:.3f} / {lat[logn][k]:.3f} ms"
                                     for k in times[logn]) + f" -> {tp_table[logn]} / {lat_table[logn]}", flush=True)
    write_header(tp_table, lat_table, times, lat, args.slices, args.chunk, args.steps,
                 torch.cuda.get_device_name(0))
    print(f"wrote {HEADER}")


if __name__ == "__main__":
    main()

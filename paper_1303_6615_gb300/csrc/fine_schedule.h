// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedules of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs.
// Measured on NVIDIA GB300, 64 steps, median of 3, ms: a sweep of 512 slices (throughput)
// / of 16 slices (latency); the fastest of each regime is kept.
//   N =     8  1: 0.197 / 0.173  -> 1 / 1
//   N =    16  1: 0.254 / 0.241  -> 1 / 1
//   N =    32  1: 0.264 / 0.253  -> 1 / 1
//   N =    64  1: 0.265 / 0.255  -> 1 / 1
//   N =   128  1: 0.363 / 0.335, 2: 0.353 / 0.261  -> 2 / 2
//   N =   256  1: 0.486 / 0.336, 2: 0.412 / 0.265, 3: 0.577 / 0.519  -> 2 / 2
//   N =   512  1: 0.894 / 0.360, 2: 0.874 / 0.327, 3: 0.764 / 0.522  -> 3 / 2
//   N =  1024  1: 1.785 / 0.616, 2: 2.433 / 0.626, 3: 1.642 / 0.835  -> 3 / 1
//   N =  2048  1: 3.793 / 0.966, 3: 3.503 / 1.147  -> 3 / 1
#pragma once

namespace arp {

// contexts whose slices fill the device (at least two per SM)
constexpr int kFineScheduleF32Tp[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 3, 3, 3};
// contexts with fewer slices
constexpr int kFineScheduleF32Lat[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1};

}  // namespace arp

// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedules of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs,
// 4 = N/8 threads with radix-16 stages.
// Measured on NVIDIA GB300, 64 steps, median of 3, ms: a sweep of 512 slices (throughput)
// / of 16 slices (latency); the fastest of each regime is kept.
//   N =     8  1: 0.183 / 0.174  -> 1 / 1
//   N =    16  1: 0.246 / 0.238  -> 1 / 1
//   N =    32  1: 0.266 / 0.256  -> 1 / 1
//   N =    64  1: 0.258 / 0.249  -> 1 / 1
//   N =   128  1: 0.365 / 0.333, 2: 0.333 / 0.261  -> 2 / 2
//   N =   256  1: 0.459 / 0.339, 2: 0.410 / 0.274, 3: 0.559 / 0.508  -> 2 / 2
//   N =   512  1: 0.881 / 0.363, 2: 0.857 / 0.338, 3: 0.715 / 0.511, 4: 0.759 / 0.539  -> 3 / 2
//   N =  1024  1: 1.722 / 0.599, 2: 2.430 / 0.623, 3: 1.566 / 0.802, 4: 1.384 / 0.739  -> 4 / 1
//   N =  2048  1: 3.755 / 0.955, 3: 3.334 / 1.122, 4: 2.957 / 1.036  -> 4 / 1
#pragma once

namespace arp {

// contexts whose slices fill the device (at least two per SM)
constexpr int kFineScheduleF32Tp[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 3, 4, 4};
// contexts with fewer slices
constexpr int kFineScheduleF32Lat[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1};

}  // namespace arp

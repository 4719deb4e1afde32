// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedules of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs.
// Measured on NVIDIA GB300, 64 steps, median of 3, ms: a sweep of 512 slices (throughput)
// / of 16 slices (latency); the fastest of each regime is kept.
//   N =     8  1: 0.187 / 0.173  -> 1 / 1
//   N =    16  1: 0.251 / 0.239  -> 1 / 1
//   N =    32  1: 0.265 / 0.257  -> 1 / 1
//   N =    64  1: 0.266 / 0.253  -> 1 / 1
//   N =   128  1: 0.369 / 0.337, 2: 0.356 / 0.258  -> 2 / 2
//   N =   256  1: 0.486 / 0.342, 2: 0.454 / 0.295, 3: 0.583 / 0.527  -> 2 / 2
//   N =   512  1: 0.900 / 0.364, 2: 0.880 / 0.328, 3: 0.765 / 0.523  -> 3 / 2
//   N =  1024  1: 1.827 / 0.640, 2: 2.123 / 0.549, 3: 1.638 / 0.859  -> 3 / 2
//   N =  2048  1: 3.868 / 0.986, 3: 3.539 / 1.184  -> 3 / 1
#pragma once

namespace arp {

// contexts whose slices fill the device (at least two per SM)
constexpr int kFineScheduleF32Tp[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 3, 3, 3};
// contexts with fewer slices
constexpr int kFineScheduleF32Lat[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 1};

}  // namespace arp

// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedules of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs,
// 4 = N/8 threads with radix-16 stages.
// Measured on NVIDIA GB300, 64 steps, median of 3, ms: a sweep of 512 slices (throughput)
// / of 16 slices (latency); the fastest of each regime is kept.
//   N =     8  1: 0.184 / 0.172  -> 1 / 1
//   N =    16  1: 0.251 / 0.241  -> 1 / 1
//   N =    32  1: 0.265 / 0.255  -> 1 / 1
//   N =    64  1: 0.267 / 0.251  -> 1 / 1
//   N =   128  1: 0.368 / 0.336, 2: 0.354 / 0.259  -> 2 / 2
//   N =   256  1: 0.477 / 0.336, 2: 0.414 / 0.266, 3: 0.581 / 0.521  -> 2 / 2
//   N =   512  1: 0.897 / 0.364, 2: 0.876 / 0.330, 3: 0.762 / 0.524, 4: 0.822 / 0.576  -> 3 / 2
//   N =  1024  1: 1.786 / 0.615, 2: 2.435 / 0.626, 3: 1.641 / 0.836, 4: 1.463 / 0.774  -> 4 / 1
//   N =  2048  1: 3.794 / 0.971, 3: 3.511 / 1.154, 4: 3.106 / 1.034  -> 4 / 1
#pragma once

namespace arp {

// contexts whose slices fill the device (at least two per SM)
constexpr int kFineScheduleF32Tp[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 3, 4, 4};
// contexts with fewer slices
constexpr int kFineScheduleF32Lat[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1};

}  // namespace arp

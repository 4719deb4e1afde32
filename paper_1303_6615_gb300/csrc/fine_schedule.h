// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedule of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs.
// Measured on NVIDIA GB300: one sweep of 512 slices x 64 steps, median of 3, ms:
//   N =     8  1: 0.216  -> 1
//   N =    16  1: 0.251  -> 1
//   N =    32  1: 0.261  -> 1
//   N =    64  1: 0.302  -> 1
//   N =   128  1: 0.440, 2: 0.376  -> 2
//   N =   256  1: 0.509, 2: 0.434, 3: 0.716  -> 2
//   N =   512  1: 0.981, 2: 0.905, 3: 1.146  -> 2
//   N =  1024  1: 1.934, 2: 2.200, 3: 1.843  -> 3
//   N =  2048  1: 4.085, 3: 3.947  -> 3
#pragma once

namespace arp {

constexpr int kFineScheduleF32[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 3, 3};

}  // namespace arp

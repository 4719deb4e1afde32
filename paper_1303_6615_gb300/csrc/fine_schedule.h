// fine_schedule.h -- written by paper_1303_6615_gb300/tune.py; do not edit.
// Default schedule of the FP32 ETDRK4 fine sweep per log2 N (index 0..11):
// 1 = N/4 threads per slice, 2 = N/2 threads, 3 = N/8 threads with lane pairs.
// Measured on NVIDIA GB300: one sweep of 512 slices x 64 steps, median of 3, ms:
//   N =     8  1: 0.187  -> 1
//   N =    16  1: 0.251  -> 1
//   N =    32  1: 0.265  -> 1
//   N =    64  1: 0.266  -> 1
//   N =   128  1: 0.370, 2: 0.352  -> 2
//   N =   256  1: 0.490, 2: 0.448, 3: 0.582  -> 2
//   N =   512  1: 0.905, 2: 0.881, 3: 0.767  -> 3
//   N =  1024  1: 1.828, 2: 2.118, 3: 1.645  -> 3
//   N =  2048  1: 3.867, 3: 3.537  -> 3
#pragma once

namespace arp {

constexpr int kFineScheduleF32[12] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 3, 3, 3};

}  // namespace arp

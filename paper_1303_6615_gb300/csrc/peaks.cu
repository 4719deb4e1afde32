// peaks.cu -- the plain-ALU peak of this GPU, measured: a kernel of fused
// multiply-adds in independent register chains, enough resident warps to keep
// every SM's FMA pipe busy, timed with events.  bench.py reports the FP32 fine
// sweep's roofline fraction against it beside the nominal unit-count peak.
#include "context.h"

namespace arp {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread
constexpr int kIters = 4096;  // FMAs per chain

template <typename T>
__global__ void __launch_bounds__(256) fma_loop_kernel(T b, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
#pragma unroll 16
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1) out[0] = s;  // keeps the chains live; never taken for the inputs used
}

template <typename T>
arp_status measure(double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_loop_kernel<T>, 256, 0) != cudaSuccess ||
      per_sm < 1)
    return ARP_ECUDA;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return ARP_ENOMEM;
  }
  const dim3 grid(sms * per_sm * 4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const T b = (T)0.999, c = (T)1e-3;
  float ms = 0.f;
  if (err == cudaSuccess) {
    fma_loop_kernel<T><<<grid, 256, 0, s>>>(b, c, out);  // warm-up
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaEventRecord(e0, s);
  for (int r = 0; r < 5 && err == cudaSuccess; ++r) {
    fma_loop_kernel<T><<<grid, 256, 0, s>>>(b, c, out);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return ARP_ECUDA;
  const double flops = 5.0 * grid.x * 256.0 * kChains * kIters * 2.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return ARP_OK;
}

}  // namespace
}  // namespace arp

extern "C" arp_status arp_alu_peak(int precision, double* tflops, void* stream) {
  if (!tflops) return ARP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == ARP_FP64) return arp::measure<double>(tflops, s);
  if (precision == ARP_FP32) return arp::measure<float>(tflops, s);
  return ARP_EINVAL;
}

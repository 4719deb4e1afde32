// common.cuh -- complex arithmetic, table views and launch helpers shared by the
// CUDA kernels of the asymptotic parareal library (1D rotating shallow water).
#pragma once

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#endif
#include <stdint.h>

namespace arp {

template <typename T>
struct __align__(sizeof(T) * 2) cpx {
  T x, y;
};

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T x, T y) { return cpx<T>{x, y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.x, s * a.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.x, -a.y}; }
// i * a
template <typename T> __host__ __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) { return {-a.y, a.x}; }
// -i * a
template <typename T> __host__ __device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) { return {a.y, -a.x}; }
// acc + a*b
template <typename T> __host__ __device__ __forceinline__ cpx<T> fma_c(cpx<T> a, cpx<T> b, cpx<T> acc) {
  return {acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x};
}
template <typename To, typename Ti> __host__ __device__ __forceinline__ cpx<To> cvt(cpx<Ti> a) {
  return {(To)a.x, (To)a.y};
}

using cd = cpx<double>;
using cf = cpx<float>;

// Eigen-branch index a = 0, 1, 2 stands for alpha = -1, 0, +1 (omega = alpha * sigma_k).
constexpr int kBranches = 3;

// Fixed quadrature-chunk size of the time average: one CUDA block evaluates the
// nonlinearity at this many consecutive nodes s_m and sums them in order; the
// chunk sums are then added in chunk order.  Fixed so that results do not
// depend on the batch size.
constexpr int kQuadChunk = 2;

// Per-wavenumber constants of L's eigenvectors (Sec. 6.1), sigma_k = sqrt(1 + k^2/F):
//   inv_sig[k] = 1/sigma_k, sk_sig[k] = F^-1/2 k / sigma_k.
template <typename T>
struct EigenView {
  const T* inv_sig;
  const T* sk_sig;
};

// ETDRK4 coefficient tables, each [3][K+1] complex (branch-major):
// E = e^{z}, E2 = e^{z/2}, Q = (h/2) phi1(z/2), f1 = h(phi1 - 3phi2 + 4phi3)(z),
// f2x2 = 2h(phi2 - 2phi3)(z), f3 = h(4phi3 - phi2)(z), z = h lambda.
template <typename T>
struct EtdView {
  const cpx<T>* E;
  const cpx<T>* E2;
  const cpx<T>* Q;
  const cpx<T>* f1;
  const cpx<T>* f2x2;
  const cpx<T>* f3;
};

// Time-average tables: phase[m][3][K+1] = e^{-i omega s_m} (complex), weight[m] = w_m.
template <typename T>
struct AvgView {
  const cpx<T>* phase;
  const T* weight;
};

}  // namespace arp

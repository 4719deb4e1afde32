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

#if defined(__CUDACC__)
// Sum and difference of two complex values for transform butterflies: FP32 as
// one packed two-lane FP32 add of the sm_100 family (__fadd2_rn), per
// component the same correctly rounded add as the scalar one, so results are
// unchanged while the instruction count halves; FP64 as two scalar adds.
// Callers use them where neither operand is a bare product, so that no
// multiply-add contraction of the scalar form is given up.
__device__ __forceinline__ cpx<float> bsum(cpx<float> a, cpx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return {r.x, r.y};
}
__device__ __forceinline__ cpx<float> bdif(cpx<float> a, cpx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  return {r.x, r.y};
}
__device__ __forceinline__ cpx<double> bsum(cpx<double> a, cpx<double> b) { return a + b; }
__device__ __forceinline__ cpx<double> bdif(cpx<double> a, cpx<double> b) { return a - b; }

// Unevaluated float pair hi + lo (|lo| <= ulp(hi)/2): about 48 significant
// bits from FP32 arithmetic, using the error-free transforms of Knuth
// (two-sum), Dekker (fast two-sum) and the FMA product error.
struct df {
  float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// (a_hi + a_lo) + b
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// (a_hi + a_lo) * (b_hi + b_lo) - (c_hi + c_lo) * (d_hi + d_lo)
__device__ __forceinline__ df df_mul_sub(df a, df b, df c, df d) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const float q = __fmul_rn(c.hi, d.hi);
  float f = __fmaf_rn(c.hi, d.hi, -q);
  f = __fmaf_rn(c.hi, d.lo, __fmaf_rn(c.lo, d.hi, f));
  df s = two_sum(p, -q);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(e, f)));
}
// complex pair arithmetic: z = (re, im) with each part a df
struct cdf {
  df re, im;
};
// (E_hi + E_lo) * (u_hi + u_lo), complex
__device__ __forceinline__ cdf cdf_mul(cf eh, cf el, cf uh, cf ul) {
  const df er{eh.x, el.x}, ei{eh.y, el.y}, ur{uh.x, ul.x}, ui{uh.y, ul.y};
  const df nei{-ei.hi, -ei.lo};
  return {df_mul_sub(er, ur, ei, ui), df_mul_sub(er, ui, nei, ur)};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cf b) { return {df_add_f(a.re, b.x), df_add_f(a.im, b.y)}; }
#endif

// Eigen-branch index a = 0, 1, 2 stands for alpha = -1, 0, +1 (omega = alpha * sigma_k).
constexpr int kBranches = 3;

// The time average splits its M nodes into chunks of ceil(M / kMaxNodeBlocks)
// consecutive nodes, one CUDA block per chunk; kMaxNodeBlocks is the SM count
// of a GB300, so the persistent chain kernel keeps one block per SM.
constexpr int kMaxNodeBlocks = 152;

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

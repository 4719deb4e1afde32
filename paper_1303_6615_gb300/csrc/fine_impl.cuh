// fine_impl.cuh -- the fine propagator F over one slice: `steps` ETDRK4 steps
// (Cox & Matthews; the fine integrator named in Sec. 6.2) of
//     da/dt = lambda a + R^H N(R a),  lambda = -i omega/eps - nu k^4,
// in L's eigen coordinates a (Sec. 6.1), where the stiff linear part is exact:
//     a1 = E2 u + Q N(u)
//     a2 = E2 u + Q N(a1)
//     a3 = E2 a1 + Q (2 N(a2) - N(u))
//     u+ = E u + f1 N(u) + 2 f2 (N(a1) + N(a2)) + f3 N(a3).
//
// One CUDA block per state.  The state's mode arrays (u, N(u), a1 and the
// running sum of the update) and the two FFT lanes stay on chip (shared
// memory, or registers in the FP32 register-resident sweep) for the whole
// sweep; only the input and output states touch global memory.
// After each transform a single pass over wavenumbers unpacks N, applies the
// ETDRK4 combination for the stage, and packs the next stage's input.
//
// SCHEME 1 instead runs integrating-factor RK4 (the comparator of Sec. 6.2):
// classical RK4 on v = e^{-t lambda} a, with the same tables E, E2:
//     x2 = E2 (u + h/2 N(u));  x3 = E2 u + h/2 N(x2);  x4 = E u + h E2 N(x3)
//     u+ = E u + h/6 (E N(u) + 2 E2 (N(x2) + N(x3)) + N(x4)).
//
// FP32 path: transforms, products, stage values a1..a3 and the N(.) terms are
// FP32, but the state u is carried as a float pair hi + lo and multiplied by
// E = e^{h lambda} held as a float pair too, so the exact linear propagation
// (a pure phase and decay per mode) does not pick up a rounding error every
// step.  For ETDRK4 the four O(h) terms of the update are summed in FP32 and
// added to the float-pair E u once per step; integrating-factor RK4 keeps its
// update sum as a float pair.  Only the N-evaluation input uses u_hi.
#pragma once

#include <type_traits>

#include "context.h"
#include "fine_schedule.h"
#include "spectral.cuh"
#include "spectral16.cuh"

namespace arp {

template <typename T> __device__ __forceinline__ cpx<T> ldgc(const cpx<T>* p);
template <> __device__ __forceinline__ cd ldgc<double>(const cd* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
template <> __device__ __forceinline__ cf ldgc<float>(const cf* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

template <typename T>
struct FineTabs {
  EtdView<T> etd;
  const cf* E_lo;  // FP32 path: low part of E, [3][K1]
  const cf* etdc;  // FP32 path: compact tables, [7][K1] complex (alpha = +1) then [7][K1] float (alpha = 0)
  const cpx<T>* tw;
  const cf* tw16;  // FP32 path, 512 <= N <= 2048: the radix-16 plan's twiddles
  const T* is;
  const T* ss;
  const double* is64;
  const double* ss64;
  double h;        // the step (integrating-factor RK4 weights)
};

// Fine time-stepping schemes sharing the four-evaluation step structure.
constexpr int kSchemeEtdrk4 = 0;
constexpr int kSchemeIfrk4 = 1;

template <int LOGN> struct FineBlock {
  static constexpr int N = 1 << LOGN;
  static constexpr int value = N / 4 < 32 ? 32 : (N / 4 > 512 ? 512 : N / 4);
};

// Second block size of the FP32 fine sweep: N/2 threads (at most 512).
template <int LOGN> struct FineBlockAlt {
  static constexpr int N = 1 << LOGN;
  static constexpr int value = N / 2 < 32 ? 32 : (N / 2 > 512 ? 512 : N / 2);
};

// Third schedule of the FP32 ETDRK4 sweep (N >= 256): N/8 threads, each
// butterfly item covering both FFT lanes at once (radix8_stage_pairs), and
// N(u), a1 and the update sum in shared memory instead of registers, so that
// the kernel fits in 128 registers and up to four slices share an SM.
template <int LOGN> struct FinePairBlock {
  static constexpr int value = (1 << LOGN) / 8;
};
__host__ __device__ constexpr bool fine_pairs_available(int logn) { return logn >= 8; }

// Transform plans of the FP32 sweep: radix-8 stages on one lane per item (the
// N/4 and N/2 schedules, state in registers); radix-8 stages on both lanes per
// item (the lane-pair schedule); radix-16 outer stages on one lane per item
// (spectral16.cuh, 512 <= N <= 2048, N/8 threads).  The last two keep N(u),
// a1 and the update sum in shared memory.
constexpr int kPlanRadix8 = 0;
constexpr int kPlanPairs = 1;
constexpr int kPlanRadix16 = 2;

template <typename T>
constexpr int fine_mode_arrays() {
  return std::is_same<T, float>::value ? 5 : 4;  // u, N(u), a1, acc (+ u_lo)
}

// Shared memory of one state's transform: two lanes and the twiddle tables.
template <typename T>
constexpr int lanes_and_twiddles(int logn) {
  return 2 * padded_len<T>(1 << logn) + twiddle_count(logn);
}

// Shared-memory layout of the fine sweep; the twiddle tables move to global
// memory (read through L1) when they would not fit (FP64 at N = 2048).
template <typename T, int LOGN>
struct FineLayout {
  static constexpr int K1 = ((1 << LOGN) - 1) / 3 + 1;
  static constexpr size_t kWithTw = (size_t)(lanes_and_twiddles<T>(LOGN) + 3 * fine_mode_arrays<T>() * K1) *
                                        sizeof(cpx<T>) + (size_t)2 * K1 * sizeof(T);
  static constexpr bool kTwShared = kWithTw <= 227 * 1024;
  static constexpr size_t kBytes = kTwShared ? kWithTw : kWithTw - (size_t)twiddle_count(LOGN) * sizeof(cpx<T>);
};

// Reads state b of a physical FP64 buffer [batch][3][H] and returns its eigen
// amplitudes at wavenumber k (k = 0 coefficients taken as real).
__device__ __forceinline__ void load_eigen64(const cd* __restrict__ src, int H, int k, double is, double ss, cd a[3]) {
  cd u[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    u[f] = src[f * H + k];
    if (k == 0) u[f].y = 0.0;
  }
  phys_to_eigen<double>(u, is, ss, a);
}

// Writes eigen amplitudes a at wavenumber k as physical coefficients.
__device__ __forceinline__ void store_phys64(cd* __restrict__ dst, int H, int k, double is, double ss, const cd a[3]) {
  cd u[3];
  eigen_to_phys<double>(a, is, ss, u);
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (k == 0) u[f].y = 0.0;
    dst[f * H + k] = u[f];
  }
}

template <typename T, int LOGN, int BLOCK, int SCHEME = kSchemeEtdrk4>
__device__ __forceinline__ void fine_body(const cd* __restrict__ in, cd* __restrict__ out, int steps,
                                          const FineTabs<T>& tb, int slice) {
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kTwShared = FineLayout<T, LOGN>::kTwShared;
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  cpx<T>* TWs = Z1 + padded_len<T>(N);
  const cpx<T>* TW = kTwShared ? TWs : tb.tw;
  cpx<T>* U = TWs + (kTwShared ? twiddle_count(LOGN) : 0);
  cpx<T>* NU = U + 3 * K1;
  cpx<T>* A1 = NU + 3 * K1;
  cpx<T>* ACC = A1 + 3 * K1;
  constexpr bool kPair = std::is_same<T, float>::value;
  static_assert(!(kPair && SCHEME != kSchemeEtdrk4), "the FP32 schemes run in fine_f32_body");
  cpx<T>* ULO = ACC + 3 * K1;                       // FP32 path only
  T* IS = reinterpret_cast<T*>(ACC + 3 * K1 + (kPair ? 3 * K1 : 0));
  T* SS = IS + K1;

  const cd* src = in + (size_t)slice * 3 * H;
  if (kTwShared)
    for (int t = threadIdx.x; t < twiddle_count(LOGN); t += BLOCK) TWs[t] = tb.tw[t];
  for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK) {
    if (k <= K) {
      const T is = tb.is[k], ss = tb.ss[k];
      IS[k] = is;
      SS[k] = ss;
      cd a[3];
      load_eigen64(src, H, k, tb.is64[k], tb.ss64[k], a);
      cpx<T> at[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        at[q] = cvt<T>(a[q]);
        U[q * K1 + k] = at[q];
        if constexpr (kPair) ULO[q * K1 + k] = cvt<float>(a[q] - cvt<double>(at[q]));
      }
      pack_mode<T, N>(Z0, Z1, k, at, is, ss);
    } else {
      zero_mode<T, N>(Z0, Z1, k);
    }
  }
  __syncthreads();

  const EtdView<T> e = tb.etd;
#pragma unroll 1
  for (int step = 0; step < steps; ++step) {
    const bool last = (step == steps - 1);
#pragma unroll 1
    for (int stage = 0; stage < 4; ++stage) {
      nonlinear_transform<T, LOGN, BLOCK>(Z0, 1, TW);  // lanes Z0, Z1 = Z0 + padded_len
      const bool pack_next = !(last && stage == 3);
      for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK) {
        if (k > K) {
          if (pack_next) zero_mode<T, N>(Z0, Z1, k);
          continue;
        }
        const T is = IS[k], ss = SS[k];
        cpx<T> bn[3], nx[3];
        unpack_mode<T, N>(Z0, Z1, k, is, ss, bn);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int i = q * K1 + k;
          if constexpr (kPair) {
            // as etd32_stage, with the state in shared memory
            if (stage == 0) {
              const cf u = U[i];
              NU[i] = bn[q];
              ACC[i] = ldgc(e.f1 + i) * bn[q];
              const cf a = ldgc(e.E2 + i) * u + ldgc(e.Q + i) * bn[q];
              A1[i] = a;
              nx[q] = a;
            } else if (stage == 3) {
              const cdf s = cdf_add(cdf_mul(ldgc(e.E + i), ldgc(tb.E_lo + i), U[i], ULO[i]),
                                    ACC[i] + ldgc(e.f3 + i) * bn[q]);
              U[i] = mk<float>(s.re.hi, s.im.hi);
              ULO[i] = mk<float>(s.re.lo, s.im.lo);
              nx[q] = U[i];
            } else {
              ACC[i] = ACC[i] + ldgc(e.f2x2 + i) * bn[q];
              nx[q] = (stage == 1) ? ldgc(e.E2 + i) * U[i] + ldgc(e.Q + i) * bn[q]
                                   : ldgc(e.E2 + i) * A1[i] + ldgc(e.Q + i) * ((T)2 * bn[q] - NU[i]);
            }
          } else if constexpr (SCHEME == kSchemeIfrk4) {
            const T h = (T)tb.h;
            if (stage == 0) {
              const cpx<T> u = U[i], E = ldgc(e.E + i);
              ACC[i] = E * u + (h / (T)6) * (E * bn[q]);
              nx[q] = ldgc(e.E2 + i) * (u + ((T)0.5 * h) * bn[q]);
            } else if (stage == 3) {
              const cpx<T> u = ACC[i] + (h / (T)6) * bn[q];
              U[i] = u;
              nx[q] = u;
            } else {
              const cpx<T> E2 = ldgc(e.E2 + i), t = E2 * bn[q];
              ACC[i] = ACC[i] + (h / (T)3) * t;
              nx[q] = (stage == 1) ? E2 * U[i] + ((T)0.5 * h) * bn[q] : ldgc(e.E + i) * U[i] + h * t;
            }
          } else {
            if (stage == 0) {
              const cpx<T> u = U[i];
              NU[i] = bn[q];
              const cpx<T> a = ldgc(e.E2 + i) * u + ldgc(e.Q + i) * bn[q];
              A1[i] = a;
              ACC[i] = ldgc(e.E + i) * u + ldgc(e.f1 + i) * bn[q];
              nx[q] = a;
            } else if (stage == 1) {
              ACC[i] = ACC[i] + ldgc(e.f2x2 + i) * bn[q];
              nx[q] = ldgc(e.E2 + i) * U[i] + ldgc(e.Q + i) * bn[q];
            } else if (stage == 2) {
              ACC[i] = ACC[i] + ldgc(e.f2x2 + i) * bn[q];
              nx[q] = ldgc(e.E2 + i) * A1[i] + ldgc(e.Q + i) * ((T)2 * bn[q] - NU[i]);
            } else {
              const cpx<T> u = ACC[i] + ldgc(e.f3 + i) * bn[q];
              U[i] = u;
              nx[q] = u;
            }
          }
        }
        if (pack_next) pack_mode<T, N>(Z0, Z1, k, nx, is, ss);
      }
      __syncthreads();
    }
  }

  cd* dst = out + (size_t)slice * 3 * H;
  for (int k = threadIdx.x; k < H; k += BLOCK) {
    if (k <= K) {
      cd a[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        a[q] = cvt<double>(U[q * K1 + k]);
        if constexpr (kPair) a[q] = a[q] + cvt<double>(ULO[q * K1 + k]);
      }
      store_phys64(dst, H, k, tb.is64[k], tb.ss64[k], a);
    } else {
#pragma unroll
      for (int f = 0; f < 3; ++f) dst[f * H + k] = {0.0, 0.0};
    }
  }
}

template <typename T, int LOGN, int BLOCK, int SCHEME = kSchemeEtdrk4>
__global__ void __launch_bounds__(BLOCK) fine_sweep_kernel(const cd* __restrict__ in, cd* __restrict__ out,
                                                           int steps, FineTabs<T> tb) {
  fine_body<T, LOGN, BLOCK, SCHEME>(in, out, steps, tb, blockIdx.x);
}

// FP32 fine sweep with the ETDRK4 state in registers: thread t owns the
// wavenumbers k = t + r BLOCK (r < MPT), holding u (float pair), N(u), a1 and
// the update sum (FP32 for ETDRK4, a float pair for integrating-factor RK4) for
// the three branches; shared memory holds only the two FFT lanes, the twiddle
// tables and the eigenvector constants.
template <int LOGN, int BLOCK, int PLAN = kPlanRadix8>
struct F32Layout {
  static constexpr int K1 = ((1 << LOGN) - 1) / 3 + 1;
  static constexpr int kMPT = (K1 + BLOCK - 1) / BLOCK;
  static constexpr bool kSmemState = PLAN != kPlanRadix8;  // N(u), a1, acc in shared memory, [3][3][K1]
  static constexpr int kTwiddles = PLAN == kPlanRadix16 ? twiddle16_count(LOGN) : twiddle_count(LOGN);
  static constexpr size_t kBytes = (size_t)(2 * padded_len<float>(1 << LOGN) + kTwiddles) * sizeof(cf) +
                                   (size_t)2 * K1 * sizeof(float) + (kSmemState ? (size_t)9 * K1 * sizeof(cf) : 0);
};

// One ETDRK4 stage of the FP32 path for one (wavenumber, branch) entry i of the
// tables: given N of the stage's input (bn), update N(u), a1 and the stage sum
// acc, at the last stage the float-pair state u/ulo, and return the next
// stage's input.  The large term E u is formed once per step, at the last
// stage (u is unchanged until then), from E and u both held as float pairs;
// the four O(h) terms f1 N(u) + f2x2 N(a) + f2x2 N(b) + f3 N(c) are summed in
// FP32 and added to it in float-pair arithmetic.  Shared by the
// register-resident sweep and the lock-step DFT-GEMM sweep so both apply the
// same arithmetic.
__device__ __forceinline__ cf etd32_stage(int stage, int i, cf bn, cf& u, cf& ulo, cf& nu, cf& a1, cf& acc,
                                          const EtdView<float>& e, const cf* __restrict__ E_lo) {
  if (stage == 0) {
    nu = bn;
    acc = ldgc(e.f1 + i) * bn;
    a1 = ldgc(e.E2 + i) * u + ldgc(e.Q + i) * bn;
    return a1;
  } else if (stage == 3) {
    const cdf s = cdf_add(cdf_mul(ldgc(e.E + i), ldgc(E_lo + i), u, ulo), acc + ldgc(e.f3 + i) * bn);
    u = mk<float>(s.re.hi, s.im.hi);
    ulo = mk<float>(s.re.lo, s.im.lo);
    return u;
  } else {
    acc = acc + ldgc(e.f2x2 + i) * bn;
    return (stage == 1) ? ldgc(e.E2 + i) * u + ldgc(e.Q + i) * bn
                        : ldgc(e.E2 + i) * a1 + ldgc(e.Q + i) * (2.0f * bn - nu);
  }
}

// The FP32 ETDRK4 stage of etd32_stage for all three branches of wavenumber k
// at once, from the compact tables: the alpha = -1 coefficients are the
// conjugates of alpha = +1's and those of alpha = 0 are real (the tables are
// built that way), so one complex entry serves two branches and the alpha = 0
// branch multiplies by real scalars.  N(u), a1 and the stage sum of branch q
// are nu[q * sq], a1[q * sq], acc[q * sq].
__device__ __forceinline__ void etd32_stage3(int stage, int k, int K1, const cf bn[3], cf u[3], cf ulo[3], cf* nu,
                                             cf* a1, cf* acc, int sq, const cf* __restrict__ cp, cf nx[3]) {
  const float* __restrict__ cz = reinterpret_cast<const float*>(cp + 7 * K1);
  enum { kE = 0, kE2, kQ, kF1, kF2x2, kF3, kElo };
  auto P = [&](int j) { return ldgc(cp + j * K1 + k); };
  auto Z = [&](int j) { return __ldg(cz + j * K1 + k); };
  auto rs = [](float r, cf x) { return mk<float>(r * x.x, r * x.y); };
  if (stage == 0) {
    const cf f1 = P(kF1), E2 = P(kE2), Q = P(kQ);
    const float f1r = Z(kF1), E2r = Z(kE2), Qr = Z(kQ);
#pragma unroll
    for (int q = 0; q < 3; q += 2) {
      const cf f = q ? f1 : conj(f1), e2 = q ? E2 : conj(E2), qq = q ? Q : conj(Q);
      nu[q * sq] = bn[q];
      acc[q * sq] = f * bn[q];
      nx[q] = a1[q * sq] = e2 * u[q] + qq * bn[q];
    }
    nu[sq] = bn[1];
    acc[sq] = rs(f1r, bn[1]);
    nx[1] = a1[sq] = rs(E2r, u[1]) + rs(Qr, bn[1]);
  } else if (stage == 3) {
    const cf E = P(kE), El = P(kElo), f3 = P(kF3);
    const float Er = Z(kE), Elr = Z(kElo), f3r = Z(kF3);
#pragma unroll
    for (int q = 0; q < 3; q += 2) {
      const cf e = q ? E : conj(E), el = q ? El : conj(El), f = q ? f3 : conj(f3);
      const cdf s = cdf_add(cdf_mul(e, el, u[q], ulo[q]), acc[q * sq] + f * bn[q]);
      u[q] = mk<float>(s.re.hi, s.im.hi);
      ulo[q] = mk<float>(s.re.lo, s.im.lo);
      nx[q] = u[q];
    }
    // alpha = 0: E real, so each component is a float-pair product by the same real pair
    const cf t = acc[sq] + rs(f3r, bn[1]);
    const df er{Er, Elr};
    const df re = df_add_f(df_mul_sub(er, df{u[1].x, ulo[1].x}, df{0.0f, 0.0f}, df{0.0f, 0.0f}), t.x);
    const df im = df_add_f(df_mul_sub(er, df{u[1].y, ulo[1].y}, df{0.0f, 0.0f}, df{0.0f, 0.0f}), t.y);
    u[1] = mk<float>(re.hi, im.hi);
    ulo[1] = mk<float>(re.lo, im.lo);
    nx[1] = u[1];
  } else {
    const cf f2 = P(kF2x2), E2 = P(kE2), Q = P(kQ);
    const float f2r = Z(kF2x2), E2r = Z(kE2), Qr = Z(kQ);
#pragma unroll
    for (int q = 0; q < 3; q += 2) {
      const cf f = q ? f2 : conj(f2), e2 = q ? E2 : conj(E2), qq = q ? Q : conj(Q);
      acc[q * sq] = acc[q * sq] + f * bn[q];
      nx[q] = (stage == 1) ? e2 * u[q] + qq * bn[q] : e2 * a1[q * sq] + qq * (2.0f * bn[q] - nu[q * sq]);
    }
    acc[sq] = acc[sq] + rs(f2r, bn[1]);
    nx[1] = (stage == 1) ? rs(E2r, u[1]) + rs(Qr, bn[1]) : rs(E2r, a1[sq]) + rs(Qr, 2.0f * bn[1] - nu[sq]);
  }
}

template <int LOGN, int BLOCK, int SCHEME = kSchemeEtdrk4, int PLAN = kPlanRadix8>
__device__ __forceinline__ void fine_f32_body(const cd* __restrict__ in, cd* __restrict__ out, int steps,
                                              const FineTabs<float>& tb, int slice) {
  static_assert(PLAN == kPlanRadix8 || SCHEME == kSchemeEtdrk4, "the shared-state schedules run ETDRK4");
  static_assert(PLAN != kPlanRadix16 || r16_available(LOGN), "the radix-16 plan covers 512 <= N <= 2048");
  using T = float;
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  constexpr bool R16 = PLAN == kPlanRadix16;
  using L = F32Layout<LOGN, BLOCK, PLAN>;
  constexpr int MPT = L::kMPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* Z0 = reinterpret_cast<cf*>(smem_raw);
  cf* Z1 = Z0 + padded_len<T>(N);
  cf* TW = Z1 + padded_len<T>(N);
  T* IS = reinterpret_cast<T*>(TW + L::kTwiddles);
  T* SS = IS + K1;
  constexpr bool kSmemState = L::kSmemState;
  cf* NUS = reinterpret_cast<cf*>(SS + K1);  // kSmemState: N(u), a1, acc in shared memory, [3][3][K1]

  cf u[MPT][3], ulo[MPT][3], nu[MPT][3], a1[MPT][3], acc[MPT][3], acclo[MPT][3];
  const cd* src = in + (size_t)slice * 3 * H;
  const cf* twg = R16 ? tb.tw16 : tb.tw;
  for (int t = threadIdx.x; t < L::kTwiddles; t += BLOCK) TW[t] = twg[t];
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k <= K) {
      const T is = tb.is[k], ss = tb.ss[k];
      IS[k] = is;
      SS[k] = ss;
      cd a[3];
      load_eigen64(src, H, k, tb.is64[k], tb.ss64[k], a);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        u[r][q] = cvt<float>(a[q]);
        ulo[r][q] = cvt<float>(a[q] - cvt<double>(u[r][q]));
      }
      pack_mode<T, N, R16>(Z0, Z1, k, u[r], is, ss);
    }
  }
  for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK)
    if (k > K) zero_mode<T, N, R16>(Z0, Z1, k);
  __syncthreads();

  const EtdView<T> e = tb.etd;
#pragma unroll 1
  for (int step = 0; step < steps; ++step) {
    const bool last = (step == steps - 1);
#pragma unroll 1
    for (int stage = 0; stage < 4; ++stage) {
      if constexpr (PLAN == kPlanRadix16)
        nonlinear_transform16<LOGN, BLOCK>(Z0, TW);  // lanes Z0, Z1 = Z0 + N
      else if constexpr (PLAN == kPlanPairs)
        nonlinear_transform_pairs<T, LOGN, BLOCK>(Z0, 1, TW);  // lanes Z0, Z1 = Z0 + padded_len
      else
        nonlinear_transform<T, LOGN, BLOCK>(Z0, 1, TW);
      const bool pack_next = !(last && stage == 3);
#pragma unroll
      for (int r = 0; r < MPT; ++r) {
        const int k = threadIdx.x + r * BLOCK;
        if (k > K) continue;
        const T is = IS[k], ss = SS[k];
        cf bn[3], nx[3];
        unpack_mode<T, N, R16>(Z0, Z1, k, is, ss, bn);
        if constexpr (SCHEME == kSchemeEtdrk4) {
          if constexpr (kSmemState)
            etd32_stage3(stage, k, K1, bn, u[r], ulo[r], NUS + k, NUS + 3 * K1 + k, NUS + 6 * K1 + k, K1, tb.etdc, nx);
          else
            etd32_stage3(stage, k, K1, bn, u[r], ulo[r], nu[r], a1[r], acc[r], 1, tb.etdc, nx);
        }
#pragma unroll
        for (int q = 0; q < 3 && SCHEME == kSchemeIfrk4; ++q) {
          const int i = q * K1 + k;
          if constexpr (SCHEME == kSchemeIfrk4) {
            const float h = (float)tb.h;
            if (stage == 0) {
              // acc = E u (float pair) + h/6 E N(u); next: E2 (u + h/2 N(u))
              const cf E = ldgc(e.E + i);
              const cdf s = cdf_add(cdf_mul(E, ldgc(tb.E_lo + i), u[r][q], ulo[r][q]), (h / 6.0f) * (E * bn[q]));
              acc[r][q] = mk<float>(s.re.hi, s.im.hi);
              acclo[r][q] = mk<float>(s.re.lo, s.im.lo);
              nx[q] = ldgc(e.E2 + i) * (u[r][q] + (0.5f * h) * bn[q]);
            } else if (stage == 3) {
              const cf t = (h / 6.0f) * bn[q];
              const df re = df_add_f(df{acc[r][q].x, acclo[r][q].x}, t.x);
              const df im = df_add_f(df{acc[r][q].y, acclo[r][q].y}, t.y);
              u[r][q] = mk<float>(re.hi, im.hi);
              ulo[r][q] = mk<float>(re.lo, im.lo);
              nx[q] = u[r][q];
            } else {
              const cf E2 = ldgc(e.E2 + i), w = E2 * bn[q];
              const cf t = (h / 3.0f) * w;
              const df re = df_add_f(df{acc[r][q].x, acclo[r][q].x}, t.x);
              const df im = df_add_f(df{acc[r][q].y, acclo[r][q].y}, t.y);
              acc[r][q] = mk<float>(re.hi, im.hi);
              acclo[r][q] = mk<float>(re.lo, im.lo);
              nx[q] = (stage == 1) ? E2 * u[r][q] + (0.5f * h) * bn[q] : ldgc(e.E + i) * u[r][q] + h * w;
            }
          }
        }
        if (pack_next) pack_mode<T, N, R16>(Z0, Z1, k, nx, is, ss);
      }
      if (pack_next)
        // bins above the kept modes, cleared by the threads whose own wavenumber lies there
        for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK)
          if (k > K) zero_mode<T, N, R16>(Z0, Z1, k);
      __syncthreads();
    }
  }

  cd* dst = out + (size_t)slice * 3 * H;
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k > K) continue;
    cd a[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) a[q] = cvt<double>(u[r][q]) + cvt<double>(ulo[r][q]);
    store_phys64(dst, H, k, tb.is64[k], tb.ss64[k], a);
  }
  for (int k = K1 + threadIdx.x; k < H; k += BLOCK) {
#pragma unroll
    for (int f = 0; f < 3; ++f) dst[f * H + k] = {0.0, 0.0};
  }
}

template <int LOGN, int BLOCK, int SCHEME = kSchemeEtdrk4>
__global__ void __launch_bounds__(BLOCK) fine_sweep_kernel_f32(const cd* __restrict__ in, cd* __restrict__ out,
                                                               int steps, FineTabs<float> tb) {
  fine_f32_body<LOGN, BLOCK, SCHEME>(in, out, steps, tb, blockIdx.x);
}

// The lane-pair schedule: at most 128 registers, so that four blocks of N/8
// threads fit an SM by registers.
template <int LOGN>
constexpr int fine_pairs_min_blocks() {
  return 65536 / (FinePairBlock<LOGN>::value * 128) < 4 ? 65536 / (FinePairBlock<LOGN>::value * 128) : 4;
}
template <int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK, fine_pairs_min_blocks<LOGN>())
    fine_sweep_kernel_f32_pairs(const cd* __restrict__ in, cd* __restrict__ out, int steps, FineTabs<float> tb) {
  fine_f32_body<LOGN, BLOCK, kSchemeEtdrk4, kPlanPairs>(in, out, steps, tb, blockIdx.x);
}

// The radix-16 schedule: N/8 threads as the lane-pair schedule, and its register bound.
template <int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK, fine_pairs_min_blocks<LOGN>())
    fine_sweep_kernel_f32_r16(const cd* __restrict__ in, cd* __restrict__ out, int steps, FineTabs<float> tb) {
  fine_f32_body<LOGN, BLOCK, kSchemeEtdrk4, kPlanRadix16>(in, out, steps, tb, blockIdx.x);
}

template <typename T>
FineTabs<T> fine_tabs(const arp_ctx* c);

template <>
inline FineTabs<double> fine_tabs<double>(const arp_ctx* c) {
  const int n = 3 * c->K1;
  return {{c->etd64, c->etd64 + n, c->etd64 + 2 * n, c->etd64 + 3 * n, c->etd64 + 4 * n, c->etd64 + 5 * n},
          nullptr, nullptr, c->tw64, nullptr, c->inv_sig64, c->sk_sig64, c->inv_sig64, c->sk_sig64, c->h};
}

template <>
inline FineTabs<float> fine_tabs<float>(const arp_ctx* c) {
  const int n = 3 * c->K1;
  return {{c->etd32, c->etd32 + n, c->etd32 + 2 * n, c->etd32 + 3 * n, c->etd32 + 4 * n, c->etd32 + 5 * n},
          c->E_lo32, c->etd32c, c->tw32, c->tw16_32, c->inv_sig32, c->sk_sig32, c->inv_sig64, c->sk_sig64, c->h};
}

template <typename T, int LOGN, int BLOCK, int SCHEME = kSchemeEtdrk4, int PLAN = kPlanRadix8>
arp_status launch_fine_block(arp_ctx* c, const cd* in, cd* out, int batch, int steps, cudaStream_t s) {
  constexpr bool kF32 = std::is_same<T, float>::value;
  const size_t smem = kF32 ? F32Layout<LOGN, BLOCK, PLAN>::kBytes : FineLayout<T, LOGN>::kBytes;
  const void* kern;
  if constexpr (PLAN == kPlanRadix16) kern = (const void*)fine_sweep_kernel_f32_r16<LOGN, BLOCK>;
  else if constexpr (PLAN == kPlanPairs) kern = (const void*)fine_sweep_kernel_f32_pairs<LOGN, BLOCK>;
  else if constexpr (kF32) kern = (const void*)fine_sweep_kernel_f32<LOGN, BLOCK, SCHEME>;
  else kern = (const void*)fine_sweep_kernel<T, LOGN, BLOCK, SCHEME>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "fine: shared-memory attribute");
  if constexpr (PLAN != kPlanRadix8) {
    // several such blocks per SM need the largest shared-memory carveout
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return check_cuda(c, e, "fine: shared-memory carveout");
  }
  FineTabs<T> tb = fine_tabs<T>(c);
  void* args[] = {(void*)&in, (void*)&out, &steps, &tb};
  e = cudaLaunchKernel(kern, dim3(batch), dim3(BLOCK), args, smem, s);
  return check_cuda(c, e, "fine: launch");
}

// The FP32 fine sweep's schedule: 1 = N/4 threads, 2 = N/2 threads, 3 = the
// lane-pair schedule with N/8 threads (ETDRK4, N >= 256), 4 = the radix-16
// plan with N/8 threads (ETDRK4, 512 <= N <= 2048).  ARP_OPT_FINE_BLOCK
// of context c if set, else the offline-tuned tables (fine_schedule.h, written
// by the project's tuner from timings on GB300): the throughput table when the
// context's slices fill the device (at least two per SM, so every level's fine
// work keeps the SMs busy), else the latency table (few slices per SM: the
// sweep of one slice bounds a level).  The schedules round differently in the
// last bits, so the choice is fixed per grid size and context shape rather
// than timed at run time, and a result never depends on a timing decision; a
// context keeps its schedule for every launch.  A schedule that does not
// apply falls back to the table's.
template <int LOGN, int SCHEME = kSchemeEtdrk4>
int fine_schedule_f32(const arp_ctx* c) {
  const bool fills = c->num_sms > 0 && c->slices >= 2 * c->num_sms;
  const int tuned = fills ? kFineScheduleF32Tp[LOGN] : kFineScheduleF32Lat[LOGN];
  const bool etd = SCHEME == kSchemeEtdrk4;
  auto applies = [&](int x) {
    return x == 1 || x == 2 || (x == 3 && etd && fine_pairs_available(LOGN)) || (x == 4 && etd && r16_available(LOGN));
  };
  int v = c->fine_block != 0 ? c->fine_block : tuned;
  if (!applies(v)) v = applies(tuned) ? tuned : 1;
  if (v == 2 && FineBlock<LOGN>::value == FineBlockAlt<LOGN>::value) v = 1;
  return v;
}

template <typename T, int LOGN, int SCHEME = kSchemeEtdrk4>
arp_status launch_fine_n(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  constexpr int B0 = FineBlock<LOGN>::value, B1 = FineBlockAlt<LOGN>::value;
  if constexpr (std::is_same<T, float>::value) {
    const int v = fine_schedule_f32<LOGN, SCHEME>(c);
    if constexpr (r16_available(LOGN) && SCHEME == kSchemeEtdrk4) {
      if (v == 4)
        return launch_fine_block<T, LOGN, FinePairBlock<LOGN>::value, SCHEME, kPlanRadix16>(c, in, out, batch,
                                                                                          c->steps, s);
    }
    if constexpr (fine_pairs_available(LOGN) && SCHEME == kSchemeEtdrk4) {
      if (v == 3)
        return launch_fine_block<T, LOGN, FinePairBlock<LOGN>::value, SCHEME, kPlanPairs>(c, in, out, batch,
                                                                                        c->steps, s);
    }
    if constexpr (B0 != B1) {
      if (v == 2) return launch_fine_block<T, LOGN, B1, SCHEME>(c, in, out, batch, c->steps, s);
    }
  }
  return launch_fine_block<T, LOGN, B0, SCHEME>(c, in, out, batch, c->steps, s);
}

template <typename T, int SCHEME = kSchemeEtdrk4>
arp_status launch_fine_prec(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  switch (c->logN) {
    case 3: return launch_fine_n<T, 3, SCHEME>(c, in, out, batch, s);
    case 4: return launch_fine_n<T, 4, SCHEME>(c, in, out, batch, s);
    case 5: return launch_fine_n<T, 5, SCHEME>(c, in, out, batch, s);
    case 6: return launch_fine_n<T, 6, SCHEME>(c, in, out, batch, s);
    case 7: return launch_fine_n<T, 7, SCHEME>(c, in, out, batch, s);
    case 8: return launch_fine_n<T, 8, SCHEME>(c, in, out, batch, s);
    case 9: return launch_fine_n<T, 9, SCHEME>(c, in, out, batch, s);
    case 10: return launch_fine_n<T, 10, SCHEME>(c, in, out, batch, s);
    case 11: return launch_fine_n<T, 11, SCHEME>(c, in, out, batch, s);
    default: return fail(c, ARP_EINVAL, "fine: unsupported grid size");
  }
}

}  // namespace arp

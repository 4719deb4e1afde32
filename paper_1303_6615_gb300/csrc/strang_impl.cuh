// strang_impl.cuh -- Strang splitting (Algorithm 3) of
//     da/dt = lambda a + R^H N(R a),  lambda = -i omega/eps - nu k^4,
// in L's eigen coordinates (Sec. 6.1).  One step of size h:
//     w = e^{lambda h/2} a;  k1 = N(w);  k2 = N(w + h/2 k1);  w = w + h k2;
//     a+ = e^{lambda h/2} w
// (the nonlinear stage read as in Algorithm 2).  Consecutive half steps
// compose exactly, so a sweep of `steps` steps applies e^{lambda h/2} once at
// each end and e^{lambda h} between steps.
//
// Uses: the fine propagator of standard parareal or of the paper's fine
// solver (ARP_OPT_FINE_SCHEME), one step of size dT as standard parareal's
// coarse solver (ARP_OPT_COARSE_SCHEME) in parallel over states, and the
// serial coarse chain built from that step.
//
// One CUDA block per state, the state in registers (wavenumbers k = t + r
// BLOCK), shared memory holding only the two FFT lanes, the twiddle tables and
// the eigen constants.  FP32 path: transforms and N in FP32, the state w kept
// as a float pair and multiplied by e^{lambda h} held as a float pair (the
// same error-free transforms as the FP32 ETDRK4 sweep); the half steps at the
// ends are applied in FP64.
#pragma once

#include <type_traits>

#include "fine_impl.cuh"

namespace arp {

template <typename T>
struct StrangTabs {
  const cpx<T>* Ef;    // [3][K1] e^{lambda h} (between steps)
  const cf* Ef_lo;     // FP32 path: its low part
  const cd* Eh64;      // [3][K1] e^{lambda h/2} in FP64 (the half steps at both ends)
  const cpx<T>* tw;
  const T* is;
  const T* ss;
  const double* is64;
  const double* ss64;
  double h;
};

template <int LOGN> struct StrangBlock {
  static constexpr int N = 1 << LOGN;
  static constexpr int value = N / 2 < 32 ? 32 : (N / 2 > 512 ? 512 : N / 2);
};

template <typename T, int LOGN>
struct StrangLayout {
  static constexpr int K1 = ((1 << LOGN) - 1) / 3 + 1;
  static constexpr size_t kBytes = (size_t)lanes_and_twiddles<T>(LOGN) * sizeof(cpx<T>) + (size_t)2 * K1 * sizeof(T);
};

// One block: stage the twiddles and eigen constants of wavenumbers k <= K.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void strang_stage_consts(cpx<T>* TW, T* IS, T* SS, const StrangTabs<T>& tb) {
  constexpr int K1 = ((1 << LOGN) - 1) / 3 + 1;
  for (int t = threadIdx.x; t < twiddle_count(LOGN); t += BLOCK) TW[t] = tb.tw[t];
  for (int k = threadIdx.x; k < K1; k += BLOCK) {
    IS[k] = tb.is[k];
    SS[k] = tb.ss[k];
  }
}

// The midpoint stage of one step on the block's state w (eigen amplitudes,
// float pair on the FP32 path): k1 = N(w), k2 = N(w + h/2 k1), w += h k2.
// Entry: Z holds the packed w; exit: w updated, Z free.
template <typename T, int LOGN, int BLOCK, int MPT>
__device__ __forceinline__ void strang_stage(cpx<T>* Z0, const cpx<T>* TW, const T* IS, const T* SS,
                                             cpx<T> (&w)[MPT][3], cf (&wlo)[MPT][3], T h) {
  constexpr int N = 1 << LOGN;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  nonlinear_transform<T, LOGN, BLOCK>(Z0, 1, TW);
  cpx<T> k1[MPT][3];
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k > K) continue;
    cpx<T> x[3];
    unpack_mode<T, N>(Z0, Z1, k, IS[k], SS[k], k1[r]);
#pragma unroll
    for (int q = 0; q < 3; ++q) x[q] = w[r][q] + ((T)0.5 * h) * k1[r][q];
    pack_mode<T, N>(Z0, Z1, k, x, IS[k], SS[k]);
  }
  for (int k = K1 + threadIdx.x; k <= zero_end<N>(); k += BLOCK) zero_mode<T, N>(Z0, Z1, k);
  __syncthreads();
  nonlinear_transform<T, LOGN, BLOCK>(Z0, 1, TW);
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k > K) continue;
    cpx<T> k2[3];
    unpack_mode<T, N>(Z0, Z1, k, IS[k], SS[k], k2);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const cpx<T> t = h * k2[q];
      if constexpr (std::is_same<T, float>::value) {
        const df re = df_add_f(df{w[r][q].x, wlo[r][q].x}, t.x);
        const df im = df_add_f(df{w[r][q].y, wlo[r][q].y}, t.y);
        w[r][q] = mk<float>(re.hi, im.hi);
        wlo[r][q] = mk<float>(re.lo, im.lo);
      } else {
        w[r][q] = w[r][q] + t;
      }
    }
  }
  __syncthreads();  // every unpack read Z before it is packed again
}

// `steps` Strang steps of state `slice` of `in` into `out` (physical FP64 [3][H]).
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void strang_body(const cd* __restrict__ in, cd* __restrict__ out, int steps,
                                            const StrangTabs<T>& tb, int slice) {
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  constexpr int MPT = (K1 + BLOCK - 1) / BLOCK;
  constexpr bool kPair = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  cpx<T>* TW = Z1 + padded_len<T>(N);
  T* IS = reinterpret_cast<T*>(TW + twiddle_count(LOGN));
  T* SS = IS + K1;
  strang_stage_consts<T, LOGN, BLOCK>(TW, IS, SS, tb);

  cpx<T> w[MPT][3];
  cf wlo[MPT][3];
  const cd* src = in + (size_t)slice * 3 * H;
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k > K) continue;
    cd a[3];
    load_eigen64(src, H, k, tb.is64[k], tb.ss64[k], a);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const cd v = tb.Eh64[q * K1 + k] * a[q];  // first half step, FP64
      w[r][q] = cvt<T>(v);
      wlo[r][q] = kPair ? cvt<float>(v - cvt<double>(w[r][q])) : mk<float>(0, 0);
    }
    pack_mode<T, N>(Z0, Z1, k, w[r], tb.is[k], tb.ss[k]);
  }
  for (int k = K1 + threadIdx.x; k <= zero_end<N>(); k += BLOCK) zero_mode<T, N>(Z0, Z1, k);
  __syncthreads();

  const T h = (T)tb.h;
#pragma unroll 1
  for (int step = 0; step < steps; ++step) {
    strang_stage<T, LOGN, BLOCK, MPT>(Z0, TW, IS, SS, w, wlo, h);
    if (step == steps - 1) break;
#pragma unroll
    for (int r = 0; r < MPT; ++r) {  // two half steps between steps: e^{lambda h}
      const int k = threadIdx.x + r * BLOCK;
      if (k > K) continue;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = q * K1 + k;
        if constexpr (kPair) {
          const cdf p = cdf_mul(ldgc(tb.Ef + i), ldgc(tb.Ef_lo + i), w[r][q], wlo[r][q]);
          w[r][q] = mk<float>(p.re.hi, p.im.hi);
          wlo[r][q] = mk<float>(p.re.lo, p.im.lo);
        } else {
          w[r][q] = ldgc(tb.Ef + i) * w[r][q];
        }
      }
      pack_mode<T, N>(Z0, Z1, k, w[r], IS[k], SS[k]);
    }
    for (int k = K1 + threadIdx.x; k <= zero_end<N>(); k += BLOCK) zero_mode<T, N>(Z0, Z1, k);
    __syncthreads();
  }

  cd* dst = out + (size_t)slice * 3 * H;
#pragma unroll
  for (int r = 0; r < MPT; ++r) {
    const int k = threadIdx.x + r * BLOCK;
    if (k > K) continue;
    cd a[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cd v = cvt<double>(w[r][q]);
      if constexpr (kPair) v = v + cvt<double>(wlo[r][q]);
      a[q] = tb.Eh64[q * K1 + k] * v;  // last half step, FP64
    }
    store_phys64(dst, H, k, tb.is64[k], tb.ss64[k], a);
  }
  for (int k = K1 + threadIdx.x; k < H; k += BLOCK) {
#pragma unroll
    for (int f = 0; f < 3; ++f) dst[f * H + k] = {0.0, 0.0};
  }
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) strang_sweep_kernel(const cd* __restrict__ in, cd* __restrict__ out,
                                                             int steps, StrangTabs<T> tb) {
  strang_body<T, LOGN, BLOCK>(in, out, steps, tb, blockIdx.x);
}

// The serial coarse chain of standard parareal with the Strang coarse step
// (Sec. 6.2): g_n = S_dT(U_n), G cache G_n = g_n, U_{n+1} = g_n + V_n (V null:
// the predictor), n = 0..S-1, in one block: a link is one Strang step of one
// state, whose two evaluations of N already spread over the block.  The state
// between links is U_{n+1} itself (FP64, physical); tb.h = dT, tb.Eh64 =
// e^{lambda dT/2}.
template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) strang_chain_kernel(cd* __restrict__ U, cd* __restrict__ Gc,
                                                             const cd* __restrict__ V, int S, StrangTabs<T> tb) {
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  constexpr int MPT = (K1 + BLOCK - 1) / BLOCK;
  constexpr bool kPair = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  cpx<T>* TW = Z1 + padded_len<T>(N);
  T* IS = reinterpret_cast<T*>(TW + twiddle_count(LOGN));
  T* SS = IS + K1;
  strang_stage_consts<T, LOGN, BLOCK>(TW, IS, SS, tb);
  // truncated modes of every output are zero
  for (int t = threadIdx.x; t < S * 3 * (H - K1); t += BLOCK) {
    const int n = t / (3 * (H - K1)), r = t - n * 3 * (H - K1);
    const int f = r / (H - K1), k = K1 + r % (H - K1);
    Gc[((size_t)n * 3 + f) * H + k] = {0.0, 0.0};
    U[((size_t)(n + 1) * 3 + f) * H + k] = {0.0, 0.0};
  }
  cd wd[MPT][3];  // FP64 w of the current link
#pragma unroll 1
  for (int n = 0; n < S; ++n) {
    cpx<T> w[MPT][3];
    cf wlo[MPT][3];
#pragma unroll
    for (int r = 0; r < MPT; ++r) {
      const int k = threadIdx.x + r * BLOCK;
      if (k > K) continue;
      cd a[3];
      load_eigen64(U + (size_t)n * 3 * H, H, k, tb.is64[k], tb.ss64[k], a);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        wd[r][q] = tb.Eh64[q * K1 + k] * a[q];
        w[r][q] = cvt<T>(wd[r][q]);
        wlo[r][q] = kPair ? cvt<float>(wd[r][q] - cvt<double>(w[r][q])) : mk<float>(0, 0);
      }
      pack_mode<T, N>(Z0, Z1, k, w[r], IS[k], SS[k]);
    }
    for (int k = K1 + threadIdx.x; k <= zero_end<N>(); k += BLOCK) zero_mode<T, N>(Z0, Z1, k);
    __syncthreads();
    strang_stage<T, LOGN, BLOCK, MPT>(Z0, TW, IS, SS, w, wlo, (T)tb.h);
#pragma unroll
    for (int r = 0; r < MPT; ++r) {
      const int k = threadIdx.x + r * BLOCK;
      if (k > K) continue;
      cd g[3], u[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cd v = cvt<double>(w[r][q]);
        if constexpr (kPair) v = v + cvt<double>(wlo[r][q]);
        g[q] = tb.Eh64[q * K1 + k] * v;
      }
      eigen_to_phys<double>(g, tb.is64[k], tb.ss64[k], u);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (k == 0) u[f].y = 0.0;
        Gc[((size_t)n * 3 + f) * H + k] = u[f];
        U[((size_t)(n + 1) * 3 + f) * H + k] = V ? u[f] + V[((size_t)n * 3 + f) * H + k] : u[f];
      }
    }
    __syncthreads();  // U_{n+1} complete before the next link reads it
  }
}

// Launchers (host side, one precision and grid size).
template <typename T, int LOGN>
arp_status launch_strang_sweep_n(arp_ctx* c, const cd* in, cd* out, int batch, int steps, const StrangTabs<T>& tb,
                                 cudaStream_t s) {
  constexpr int BLOCK = StrangBlock<LOGN>::value;
  const size_t smem = StrangLayout<T, LOGN>::kBytes;
  const void* kern = (const void*)strang_sweep_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "strang: shared-memory attribute");
  void* args[] = {(void*)&in, (void*)&out, &steps, (void*)&tb};
  return check_cuda(c, cudaLaunchKernel(kern, dim3(batch), dim3(BLOCK), args, smem, s), "strang: launch");
}

template <typename T, int LOGN>
arp_status launch_strang_chain_n(arp_ctx* c, cd* U, cd* Gc, const cd* V, const StrangTabs<T>& tb, cudaStream_t s) {
  constexpr int BLOCK = StrangBlock<LOGN>::value;
  const size_t smem = StrangLayout<T, LOGN>::kBytes;
  const void* kern = (const void*)strang_chain_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "strang chain: shared-memory attribute");
  int S = c->slices;
  void* args[] = {(void*)&U, (void*)&Gc, (void*)&V, &S, (void*)&tb};
  return check_cuda(c, cudaLaunchKernel(kern, dim3(1), dim3(BLOCK), args, smem, s), "strang chain: launch");
}

}  // namespace arp

// coarse_impl.cuh -- the discretised time average of the nonlinearity
// (Eq. 2.1-2.2, Algorithm 1), in L's eigen coordinates:
//     Nbar(a)_k = sum_{m=0}^{M-1} w_m e^{+i omega_k s_m} [R^H N(R e^{-i omega s_m} a)]_k.
//
// Algorithm 1 evaluates the M terms in parallel and sums them.  Here one CUDA
// block takes one state and one chunk of consecutive nodes (the context's
// nodes-per-block count, fixed per context so results do not depend on the
// batch), evaluates the nonlinearity at each node with the state held in
// shared memory, and accumulates the weighted, back-rotated terms on chip in
// node order; a separate FP64 pass adds the chunk sums in chunk order.
// The B x M x 3 x (K+1) tensor of individual terms is never written.
#pragma once

#include "fine_impl.cuh"

namespace arp {

template <typename T>
struct NbarTabs {
  AvgView<T> avg;
  const cpx<T>* tw;
  const cf* tw16;  // FP32, 512 <= N <= 2048: the radix-16 plan's twiddles (the cluster chain)
  const T* is;
  const T* ss;
};

template <typename T>
inline size_t nbar_smem_bytes(int logn) {
  const int K1 = ((1 << logn) - 1) / 3 + 1;
  return (size_t)(lanes_and_twiddles<T>(logn) + 6 * K1) * sizeof(cpx<T>) + (size_t)2 * K1 * sizeof(T);
}

// Evaluates, for the eigen state WS (shared memory, visible to the block),
// ACC = sum_{m0 <= m < m1} w_m conj(ph_m) . b(ph_m . WS), ph_m = e^{-i omega s_m},
// in node order.  Block-uniform m0, m1; ends synchronised.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void nbar_nodes(const cpx<T>* WS, cpx<T>* ACC, int m0, int m1, const NbarTabs<T>& tb,
                                           cpx<T>* Z0, cpx<T>* Z1, const cpx<T>* TW, const T* IS, const T* SS) {
  constexpr int N = 1 << LOGN;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK) {
    if (k > K) {
      zero_mode<T, N>(Z0, Z1, k);
      continue;
    }
    cpx<T> x[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ACC[q * K1 + k] = mk<T>(0, 0);
      if (m0 < m1) x[q] = ldgc(tb.avg.phase + ((size_t)m0 * 3 + q) * K1 + k) * WS[q * K1 + k];
    }
    if (m0 < m1) pack_mode<T, N>(Z0, Z1, k, x, IS[k], SS[k]);
  }
  __syncthreads();
#pragma unroll 1
  for (int m = m0; m < m1; ++m) {
    nonlinear_transform<T, LOGN, BLOCK>(Z0, 1, TW);  // lanes Z0, Z1 = Z0 + padded_len
    const bool next = (m + 1 < m1);
    const T wm = tb.avg.weight[m];
    for (int k = threadIdx.x; k <= zero_end<N>(); k += BLOCK) {
      if (k > K) {
        if (next) zero_mode<T, N>(Z0, Z1, k);
        continue;
      }
      const T is = IS[k], ss = SS[k];
      cpx<T> bn[3], x[3];
      unpack_mode<T, N>(Z0, Z1, k, is, ss, bn);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = q * K1 + k;
        // w_m e^{+i omega s_m} = w_m conj(e^{-i omega s_m})
        const cpx<T> ph = ldgc(tb.avg.phase + ((size_t)m * 3 + q) * K1 + k);
        ACC[i] = ACC[i] + wm * (conj(ph) * bn[q]);
        if (next) x[q] = ldgc(tb.avg.phase + ((size_t)(m + 1) * 3 + q) * K1 + k) * WS[i];
      }
      if (next) pack_mode<T, N>(Z0, Z1, k, x, is, ss);
    }
    __syncthreads();
  }
}

// grid (P, batch): block (p, b) handles nodes m in [p C, min(M, (p+1) C)), C = nodes per block.
// W: eigen FP64 [batch][3][K1]; partial: eigen FP64 [batch][P][3][K1].
template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) nbar_partial_kernel(const cd* __restrict__ W, cd* __restrict__ partial,
                                                             int M, int chunk, NbarTabs<T> tb) {
  constexpr int N = 1 << LOGN;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  cpx<T>* TW = Z1 + padded_len<T>(N);
  cpx<T>* WS = TW + twiddle_count(LOGN);
  cpx<T>* ACC = WS + 3 * K1;
  T* IS = reinterpret_cast<T*>(ACC + 3 * K1);
  T* SS = IS + K1;

  const int p = blockIdx.x, b = blockIdx.y, P = gridDim.x;
  const int m0 = min(M, p * chunk);
  const int m1 = min(M, m0 + chunk);
  const cd* w = W + (size_t)b * 3 * K1;
  for (int t = threadIdx.x; t < twiddle_count(LOGN); t += BLOCK) TW[t] = tb.tw[t];
  for (int k = threadIdx.x; k < K1; k += BLOCK) {
    IS[k] = tb.is[k];
    SS[k] = tb.ss[k];
#pragma unroll
    for (int q = 0; q < 3; ++q) WS[q * K1 + k] = cvt<T>(w[q * K1 + k]);
  }
  __syncthreads();
  nbar_nodes<T, LOGN, BLOCK>(WS, ACC, m0, m1, tb, Z0, Z1, TW, IS, SS);
  cd* dst = partial + ((size_t)b * P + p) * 3 * K1;
  for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) dst[i] = cvt<double>(ACC[i]);
}

template <typename T>
NbarTabs<T> nbar_tabs(const arp_ctx* c);
template <>
inline NbarTabs<double> nbar_tabs<double>(const arp_ctx* c) {
  return {{c->phase64, c->weight64}, c->tw64, nullptr, c->inv_sig64, c->sk_sig64};
}
template <>
inline NbarTabs<float> nbar_tabs<float>(const arp_ctx* c) {
  return {{c->phase32, c->weight32}, c->tw32, c->tw16_32, c->inv_sig32, c->sk_sig32};
}

template <typename T, int LOGN>
arp_status launch_nbar_n(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  constexpr int BLOCK = FineBlock<LOGN>::value;
  const size_t smem = nbar_smem_bytes<T>(LOGN);
  auto kern = nbar_partial_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "nbar: shared-memory attribute");
  kern<<<dim3(c->P, batch), BLOCK, smem, s>>>(W, partial, c->M, c->qc, nbar_tabs<T>(c));
  return check_cuda(c, cudaGetLastError(), "nbar: launch");
}

template <typename T>
arp_status launch_nbar_prec(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  switch (c->logN) {
    case 3: return launch_nbar_n<T, 3>(c, W, partial, batch, s);
    case 4: return launch_nbar_n<T, 4>(c, W, partial, batch, s);
    case 5: return launch_nbar_n<T, 5>(c, W, partial, batch, s);
    case 6: return launch_nbar_n<T, 6>(c, W, partial, batch, s);
    case 7: return launch_nbar_n<T, 7>(c, W, partial, batch, s);
    case 8: return launch_nbar_n<T, 8>(c, W, partial, batch, s);
    case 9: return launch_nbar_n<T, 9>(c, W, partial, batch, s);
    case 10: return launch_nbar_n<T, 10>(c, W, partial, batch, s);
    case 11: return launch_nbar_n<T, 11>(c, W, partial, batch, s);
    default: return fail(c, ARP_EINVAL, "nbar: unsupported grid size");
  }
}

}  // namespace arp

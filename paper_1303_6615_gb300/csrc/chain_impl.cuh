// chain_impl.cuh -- the serial coarse chain of parareal (the second loop of
// Algorithm 4, the first term of Eq. 3.1): for n = 0..S-1,
//     g_n = G(U_n),   U_{n+1} = g_n + V_n   (V = F - G of the previous
//     iterate; absent for the predictor),
// with G the asymptotic slow solver of Algorithm 2:
//     w = e^{dT/2 D} u; k1 = Nbar(w); k2 = Nbar(w + dT/2 k1);
//     g = e^{-(dT/eps) L} e^{dT/2 D} (w + dT k2).
//
// One cooperative launch of P blocks (P = quadrature-node chunks, at most one
// block per SM), persistent across all S links.  Block j evaluates the
// nonlinearity at its nodes for both averages of a link and writes its partial
// sum; a grid barrier separates the two averages and the links.  Every block
// then sums the P partials in the same fixed order and so holds the same next
// state without a third barrier; block 0 writes g_n and U_{n+1}.
//
// The grid barrier spins on a global counter with a wall-clock limit: after
// kBarrierTimeoutNs a block records ARP_ETIMEOUT in the status word and every
// block returns, so a lost block can never hang the GPU.
#pragma once

#include "coarse_impl.cuh"

namespace arp {

constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier across the co-resident blocks of a cooperative launch.  `epoch` is
// the block's running target (gridDim.x per barrier); returns false if the
// status word is set (a timeout here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* status, unsigned& epoch, bool arrive = true) {
  __shared__ int ok;
  __threadfence();  // this thread's global writes before the block's arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += gridDim.x;
    __threadfence();
    if (arrive) atomicAdd(count, 1u);
    const unsigned long long t0 = globaltimer_ns();
    int good = 1;
    for (;;) {
      const unsigned v = *(volatile unsigned*)count;
      if ((int)(v - epoch) >= 0) break;
      if (*(volatile unsigned*)status != 0u) {
        good = 0;
        break;
      }
      if (globaltimer_ns() - t0 > kBarrierTimeoutNs) {
        atomicCAS(status, 0u, (unsigned)ARP_ETIMEOUT);
        good = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

struct ChainArgs {
  const cd* V;       // [S][3][H] or null (predictor)
  cd* U;             // [(S+1)][3][H]; U_0 read, U_1..U_S written
  cd* Gc;            // [S][3][H] written
  cd* part1;         // [P][3][K1]
  cd* part2;         // [P][3][K1]
  unsigned* count;   // grid-barrier counter, zero at launch
  unsigned* status;  // zero at launch
  int S, M, chunk;
  int skip_arrival;  // test hook: block 0 skips its first arrival
  double dT;
  const double* is64;
  const double* ss64;
  const double* dhalf;
  const cd* gphase;
};

template <typename T>
inline size_t chain_smem_bytes(int N) {
  const int K1 = (N - 1) / 3 + 1;
  return (size_t)(2 * N + N / 2 + 6 * K1) * sizeof(cpx<T>) + (size_t)2 * K1 * sizeof(T) + (size_t)3 * K1 * sizeof(cd);
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) chain_kernel(ChainArgs a, NbarTabs<T> tb) {
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* W64 = reinterpret_cast<cd*>(smem_raw);               // w of the current link, eigen FP64
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(W64 + 3 * K1);
  cpx<T>* Z1 = Z0 + N;
  cpx<T>* TW = Z1 + N;
  cpx<T>* WS = TW + N / 2;
  cpx<T>* ACC = WS + 3 * K1;
  T* IS = reinterpret_cast<T*>(ACC + 3 * K1);
  T* SS = IS + K1;

  const int j = blockIdx.x, P = gridDim.x;
  const int m0 = min(a.M, j * a.chunk);
  const int m1 = min(a.M, m0 + a.chunk);
  unsigned epoch = 0;

  for (int t = threadIdx.x; t < N / 2; t += BLOCK) TW[t] = tb.tw[t];
  for (int k = threadIdx.x; k < K1; k += BLOCK) {
    IS[k] = tb.is[k];
    SS[k] = tb.ss[k];
    cd x[3], e[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      x[f] = a.U[f * H + k];
      if (k == 0) x[f].y = 0.0;
    }
    phys_to_eigen<double>(x, a.is64[k], a.ss64[k], e);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      W64[q * K1 + k] = a.dhalf[k] * e[q];
      WS[q * K1 + k] = cvt<T>(W64[q * K1 + k]);
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int n = 0; n < a.S; ++n) {
    // first average, on w
    nbar_nodes<T, LOGN, BLOCK>(WS, ACC, m0, m1, tb, Z0, Z1, TW, IS, SS);
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) a.part1[(size_t)j * 3 * K1 + i] = cvt<double>(ACC[i]);
    if (!grid_barrier(a.count, a.status, epoch, !(a.skip_arrival && j == 0 && n == 0))) return;
    // midpoint state w + dT/2 k1, then the second average on it
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) {
      cd s = {0.0, 0.0};
      for (int p = 0; p < P; ++p) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(a.part1 + (size_t)p * 3 * K1 + i));
        s = s + cd{v.x, v.y};
      }
      WS[i] = cvt<T>(W64[i] + (0.5 * a.dT) * s);
    }
    __syncthreads();
    nbar_nodes<T, LOGN, BLOCK>(WS, ACC, m0, m1, tb, Z0, Z1, TW, IS, SS);
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) a.part2[(size_t)j * 3 * K1 + i] = cvt<double>(ACC[i]);
    if (!grid_barrier(a.count, a.status, epoch)) return;
    // g = e^{-(dT/eps)L} e^{dT/2 D}(w + dT k2); U_{n+1} = g + V_n; next w
    cd* gout = a.Gc + (size_t)n * 3 * H;
    cd* uout = a.U + (size_t)(n + 1) * 3 * H;
    const cd* v = a.V ? a.V + (size_t)n * 3 * H : nullptr;
    for (int k = threadIdx.x; k < H; k += BLOCK) {
      if (k >= K1) {
        if (j == 0) {
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            gout[f * H + k] = {0.0, 0.0};
            uout[f * H + k] = {0.0, 0.0};
          }
        }
        continue;
      }
      cd g[3], u[3], e[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = q * K1 + k;
        cd s = {0.0, 0.0};
        for (int p = 0; p < P; ++p) {
          const double2 vv = __ldcg(reinterpret_cast<const double2*>(a.part2 + (size_t)p * 3 * K1 + i));
          s = s + cd{vv.x, vv.y};
        }
        g[q] = a.dhalf[k] * (a.gphase[i] * (W64[i] + a.dT * s));
      }
      eigen_to_phys<double>(g, a.is64[k], a.ss64[k], u);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (k == 0) u[f].y = 0.0;
        if (j == 0) gout[f * H + k] = u[f];
        if (v) u[f] = u[f] + v[f * H + k];
        if (j == 0) uout[f * H + k] = u[f];
        if (k == 0) u[f].y = 0.0;
      }
      phys_to_eigen<double>(u, a.is64[k], a.ss64[k], e);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = q * K1 + k;
        W64[i] = a.dhalf[k] * e[q];
        WS[i] = cvt<T>(W64[i]);
      }
    }
    __syncthreads();
  }
}

template <typename T, int LOGN>
arp_status launch_chain_n(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  constexpr int BLOCK = FineBlock<LOGN>::value;
  const size_t smem = chain_smem_bytes<T>(1 << LOGN);
  auto kern = chain_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: shared-memory attribute");
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: occupancy");
  if ((long long)per_sm * sms < c->P) return fail(c, ARP_EINVAL, "chain: grid cannot be co-resident");
  e = cudaMemsetAsync(c->sync, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: reset");
  ChainArgs a{V, U, Gc, c->partial, c->part2, c->sync, c->sync + 1, c->slices, c->M, c->qc, c->skip_arrival, c->dT,
              c->inv_sig64, c->sk_sig64, c->dhalf, c->gphase};
  c->skip_arrival = 0;
  NbarTabs<T> tb = nbar_tabs<T>(c);
  void* args[] = {&a, &tb};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(c->P), dim3(BLOCK), args, smem, s);
  return check_cuda(c, e, "chain: cooperative launch");
}

template <typename T>
arp_status launch_chain_prec(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  switch (c->logN) {
    case 3: return launch_chain_n<T, 3>(c, U, Gc, V, s);
    case 4: return launch_chain_n<T, 4>(c, U, Gc, V, s);
    case 5: return launch_chain_n<T, 5>(c, U, Gc, V, s);
    case 6: return launch_chain_n<T, 6>(c, U, Gc, V, s);
    case 7: return launch_chain_n<T, 7>(c, U, Gc, V, s);
    case 8: return launch_chain_n<T, 8>(c, U, Gc, V, s);
    case 9: return launch_chain_n<T, 9>(c, U, Gc, V, s);
    case 10: return launch_chain_n<T, 10>(c, U, Gc, V, s);
    case 11: return launch_chain_n<T, 11>(c, U, Gc, V, s);
    default: return fail(c, ARP_EINVAL, "chain: unsupported grid size");
  }
}

}  // namespace arp

// chain_impl.cuh -- the serial coarse chain of parareal (the second loop of
// Algorithm 4, the first term of Eq. 3.1): for n = 0..S-1,
//     g_n = G(U_n),   U_{n+1} = g_n + V_n   (V = F - G of the previous
//     iterate; absent for the predictor),
// with G the asymptotic slow solver of Algorithm 2:
//     w = e^{dT/2 D} u; k1 = Nbar(w); k2 = Nbar(w + dT/2 k1);
//     g = e^{-(dT/eps) L} e^{dT/2 D} (w + dT k2).
//
// One cooperative launch of P blocks (P = quadrature-node chunks, at most one
// block per SM), persistent across all S links.  Per link:
//   A  every block evaluates the nonlinearity at its nodes for w and writes its
//      partial sum;                                              -- barrier
//   B  block j sums the P partials of its own wavenumbers (fixed order) and
//      writes the midpoint state w + dT/2 k1 for them;           -- barrier
//   C  every block reads the midpoint state, evaluates its nodes, writes the
//      partial sum;                                              -- barrier
//   D  block j sums those partials for its wavenumbers, forms g, U_{n+1} and the
//      next link's w for them;                                   -- barrier
// so the FP64 work of the epilogues (slow on this part) is spread over the
// blocks instead of repeated in each.
//
// The grid barrier spins on a global counter with a wall-clock limit: after
// kBarrierTimeoutNs a block records ARP_ETIMEOUT in the status word and every
// block returns, so a lost block can never hang the GPU.
#pragma once

#include <type_traits>

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
// status word is set (a timeout here or elsewhere).  The block barrier orders
// every thread's writes before thread 0's release-add arrival; thread 0's
// acquire loads of the counter order the block's later reads.
__device__ __forceinline__ void arrive_release(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* status, unsigned& epoch, bool arrive = true) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += gridDim.x;
    if (arrive) arrive_release(count);
    const unsigned long long t0 = globaltimer_ns();
    int good = 1;
    for (;;) {
      const unsigned v = load_acquire(count);
      if ((int)(v - epoch) >= 0) break;
      if (load_acquire(status) != 0u) {
        good = 0;
        break;
      }
      if (globaltimer_ns() - t0 > kBarrierTimeoutNs) {
        atomicCAS(status, 0u, (unsigned)ARP_ETIMEOUT);
        good = 0;
        break;
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ cd ldcg_c(const cd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

struct ChainArgs {
  const cd* V;       // [S][3][H] or null (predictor)
  cd* U;             // [(S+1)][3][H]; U_0 read, U_1..U_S written
  cd* Gc;            // [S][3][H] written
  cd* part1;         // [P][3][K1]
  cd* part2;         // [P][3][K1]
  cd* wg;            // [3][K1] w of the current link (eigen, FP64)
  cd* w2g;           // [3][K1] midpoint state
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
inline size_t chain_smem_bytes(int logn) {
  const int K1 = ((1 << logn) - 1) / 3 + 1;
  return (size_t)(lanes_and_twiddles<T>(logn) + 6 * K1) * sizeof(cpx<T>) + (size_t)2 * K1 * sizeof(T);
}

// Sums part[p][i] over p = 0..P-1 for the `count` indices i = first + r*stride...
// Each sum is split over a half-warp (lane l takes p = l, l+16, ...) and closed
// by a fixed shuffle tree, so the order of additions never changes.  Results go
// to red[r] in shared memory (visible after the caller's __syncthreads()).
template <int BLOCK>
__device__ __forceinline__ void sum_partials(const cd* part, int P, int K1x3, const int* idx, int count, cd* red) {
  const int lane = threadIdx.x & 15;
  // the trip count is the same for every thread, so all lanes reach every shuffle
  for (int it0 = 0; it0 < count; it0 += BLOCK / 16) {
    const int it = it0 + (int)(threadIdx.x >> 4);
    const bool active = it < count;
    cd s = {0.0, 0.0};
    if (active) {
      const int i = idx[it];
      for (int p = lane; p < P; p += 16) s = s + ldcg_c(part + (size_t)p * K1x3 + i);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      s.x += __shfl_down_sync(0xffffffffu, s.x, off, 16);
      s.y += __shfl_down_sync(0xffffffffu, s.y, off, 16);
    }
    if (active && lane == 0) red[it] = s;
  }
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) chain_kernel(ChainArgs a, NbarTabs<T> tb) {
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  constexpr int kMaxOwn = 64;  // own wavenumbers per block (K1 <= 683 and P >= 11 for N = 2048)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Z0 = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Z1 = Z0 + padded_len<T>(N);
  cpx<T>* TW = Z1 + padded_len<T>(N);
  cpx<T>* WS = TW + twiddle_count(LOGN);
  cpx<T>* ACC = WS + 3 * K1;
  T* IS = reinterpret_cast<T*>(ACC + 3 * K1);
  T* SS = IS + K1;
  __shared__ int own_idx[3 * kMaxOwn];
  __shared__ cd red[3 * kMaxOwn];

  const int j = blockIdx.x, P = gridDim.x;
  const int m0 = min(a.M, j * a.chunk);
  const int m1 = min(a.M, m0 + a.chunk);
  const int per = (K1 + P - 1) / P;
  const int k0 = min(K1, j * per), k1 = min(K1, k0 + per);
  const int nown = k1 - k0;  // own wavenumbers, <= kMaxOwn (checked on the host)
  unsigned epoch = 0;

  for (int t = threadIdx.x; t < twiddle_count(LOGN); t += BLOCK) TW[t] = tb.tw[t];
  for (int k = threadIdx.x; k < K1; k += BLOCK) {
    IS[k] = tb.is[k];
    SS[k] = tb.ss[k];
  }
  for (int r = threadIdx.x; r < 3 * nown; r += BLOCK) own_idx[r] = (r / nown) * K1 + k0 + r % nown;
  // initial w = e^{dT/2 D} R^H U_0 for the own wavenumbers
  for (int k = k0 + (int)threadIdx.x; k < k1; k += BLOCK) {
    cd x[3], e[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      x[f] = a.U[f * H + k];
      if (k == 0) x[f].y = 0.0;
    }
    phys_to_eigen<double>(x, a.is64[k], a.ss64[k], e);
#pragma unroll
    for (int q = 0; q < 3; ++q) a.wg[q * K1 + k] = a.dhalf[k] * e[q];
  }
  if (!grid_barrier(a.count, a.status, epoch)) return;
  for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) WS[i] = cvt<T>(ldcg_c(a.wg + i));
  __syncthreads();

#pragma unroll 1
  for (int n = 0; n < a.S; ++n) {
    // A: first average, on w
    nbar_nodes<T, LOGN, BLOCK>(WS, ACC, m0, m1, tb, Z0, Z1, TW, IS, SS);
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) a.part1[(size_t)j * 3 * K1 + i] = cvt<double>(ACC[i]);
    if (!grid_barrier(a.count, a.status, epoch, !(a.skip_arrival && j == 0 && n == 0))) return;
    // B: midpoint state w + dT/2 k1 for the own wavenumbers
    sum_partials<BLOCK>(a.part1, P, 3 * K1, own_idx, 3 * nown, red);
    __syncthreads();
    for (int r = threadIdx.x; r < 3 * nown; r += BLOCK) {
      const int i = own_idx[r];
      a.w2g[i] = ldcg_c(a.wg + i) + (0.5 * a.dT) * red[r];
    }
    if (!grid_barrier(a.count, a.status, epoch)) return;
    // C: second average, on the midpoint state
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) WS[i] = cvt<T>(ldcg_c(a.w2g + i));
    __syncthreads();
    nbar_nodes<T, LOGN, BLOCK>(WS, ACC, m0, m1, tb, Z0, Z1, TW, IS, SS);
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) a.part2[(size_t)j * 3 * K1 + i] = cvt<double>(ACC[i]);
    if (!grid_barrier(a.count, a.status, epoch)) return;
    // D: g = e^{-(dT/eps)L} e^{dT/2 D}(w + dT k2); U_{n+1} = g + V_n; next w
    sum_partials<BLOCK>(a.part2, P, 3 * K1, own_idx, 3 * nown, red);
    __syncthreads();
    cd* gout = a.Gc + (size_t)n * 3 * H;
    cd* uout = a.U + (size_t)(n + 1) * 3 * H;
    const cd* v = a.V ? a.V + (size_t)n * 3 * H : nullptr;
    for (int r = threadIdx.x; r < nown; r += BLOCK) {
      const int k = k0 + r;
      cd g[3], u[3], e[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = q * K1 + k;
        g[q] = a.dhalf[k] * (a.gphase[i] * (ldcg_c(a.wg + i) + a.dT * red[q * nown + r]));
      }
      eigen_to_phys<double>(g, a.is64[k], a.ss64[k], u);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (k == 0) u[f].y = 0.0;
        gout[f * H + k] = u[f];
        if (v) u[f] = u[f] + v[f * H + k];
        uout[f * H + k] = u[f];
      }
      phys_to_eigen<double>(u, a.is64[k], a.ss64[k], e);
#pragma unroll
      for (int q = 0; q < 3; ++q) a.wg[q * K1 + k] = a.dhalf[k] * e[q];
    }
    if (j == 0) {
      for (int t = threadIdx.x; t < 3 * (H - K1); t += BLOCK) {
        const int f = t / (H - K1), k = K1 + t % (H - K1);
        gout[f * H + k] = {0.0, 0.0};
        uout[f * H + k] = {0.0, 0.0};
      }
    }
    if (!grid_barrier(a.count, a.status, epoch)) return;
    for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) WS[i] = cvt<T>(ldcg_c(a.wg + i));
    __syncthreads();
  }
}

template <typename T, int LOGN>
arp_status launch_chain_n(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  constexpr int BLOCK = FineBlock<LOGN>::value;
  const size_t smem = chain_smem_bytes<T>(LOGN);
  const void* kern = (const void*)chain_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: shared-memory attribute");
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: occupancy");
  if ((long long)per_sm * sms < c->P) return fail(c, ARP_EINVAL, "chain: grid cannot be co-resident");
  if ((c->K1 + c->P - 1) / c->P > 64) return fail(c, ARP_EINVAL, "chain: too many wavenumbers per block");
  e = cudaMemsetAsync(c->sync, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return check_cuda(c, e, "chain: reset");
  ChainArgs a{V, U, Gc, c->partial, c->part2, c->W, c->W2, c->sync, c->sync + 1, c->slices, c->M, c->qc,
              c->skip_arrival, c->dT, c->inv_sig64, c->sk_sig64, c->dhalf, c->gphase};
  c->skip_arrival = 0;
  NbarTabs<T> tb = nbar_tabs<T>(c);
  void* args[] = {&a, &tb};
  e = cudaLaunchCooperativeKernel(kern, dim3(c->P), dim3(BLOCK), args, smem, s);
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

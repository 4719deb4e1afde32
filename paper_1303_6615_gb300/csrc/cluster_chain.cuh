// cluster_chain.cuh -- the serial coarse chain of parareal (Eq. 3.1, the second
// loop of Algorithm 4) inside one thread-block cluster:
//     g_n = G(U_n),  U_{n+1} = g_n + V_n,  n = 0..S-1,
// with G the asymptotic slow solver of Algorithm 2 (two time averages per link).
//
// C CTAs (16 where the part allows clusters that large, else 8) form one
// cluster.  CTA j owns the quadrature nodes [j q, (j+1) q), q = ceil(M/C), and
// evaluates all of them at once (two FFT lanes per node), then sums their
// weighted, back-rotated terms in node order.  The sum over CTAs, and the
// exchange of the next state, are asynchronous stores into other CTAs' shared
// memory (distributed shared memory, st.async) that each count their bytes on
// an mbarrier of the receiving CTA -- one-way signals, no cluster-wide barrier
// and no fence on the serial path, no global-memory atomics.  Per time average:
//   1  every CTA: its nodes' partial sum for the current state WS, stored
//      into the reduction buffer RED[rank] of each wavenumber's owner CTA
//   2  the owner threads wait until their CTA's RED barrier has counted the
//      C ranks' bytes
//   3  CTA j, for its own (branch, wavenumber) pairs, one thread each: the sum
//      of RED over the C ranks (fixed order), the FP64 epilogue (the midpoint
//      state, or g and the next w), and the float copy of the result stored
//      into WS of every CTA
//   4  every thread waits until its CTA's WS barrier has counted the whole
//      state (3 K1 entries); nothing reads the last link's final state, so it
//      is not sent
// Each barrier completes once per time average.  The next phase's byte count
// is posted right after a wait, before this CTA sends anything that could
// start that phase, and no phase can complete before every thread that waits
// on it has seen the previous one (a CTA's next stores depend on its waits).
// Every wait gives up after kBarrierTimeoutNs: the thread records ARP_ETIMEOUT
// in the status word, its CTA leaves the loop at the next block barrier, waits
// a bounded moment for stores in flight and meets the others at the final
// cluster barrier, whom their own bounded waits release.
// Only what the next link needs stays on this serial path, and GB300's FP64
// units (1/64 of the FP32 rate) make every FP64 instruction on it costly:
//   - the chain writes g_n = G(U_n) in the eigen basis (Ge) and leaves the
//     basis change U_{n+1} = R g_n + V_n, the G cache R g_n and the
//     truncated modes to a parallel kernel afterwards (finish_body);
//   - the next w needs no basis change either: R is unitary, so
//     e^{dT/2 D} R^H (R g + V_n) = e^{dT/2 D} g + VT_n, with
//     VT_n = e^{dT/2 D} R^H V_n formed for all links in parallel beforehand
//     (corr_body) and prefetched two links ahead.  (Before that basis change
//     the oracle also drops the rounding-level imaginary part of R g at
//     k = 0; here that projection reaches U and the G cache, not w: a
//     difference at the rounding level.)
// The FP64 state w of a wavenumber lives only in its owner CTA, so every
// exchanged copy is freshly rounded from FP64.
#pragma once

#include <cooperative_groups.h>

#include "chain_impl.cuh"  // globaltimer_ns, kBarrierTimeoutNs
#include "coarse_impl.cuh"
#include "spectral16.cuh"

namespace arp {

struct ClusterChainArgs {
  const cd* VT;      // [slices][3][K1] e^{dT/2 D} R^H V_n (eigen basis), or null (predictor: V = 0)
  const cd* U0;      // [3][H] the chain's initial state U_0 (read when Win is null)
  cd* Ge;            // [slices][3][K1] g_n = G(U_n) in the eigen basis, written
  int S, M, q, own;  // links of this launch, nodes, nodes per CTA, wavenumbers per CTA
  int ph_smem;       // node phases staged in shared memory (else read from the table)
  int tmp_smem;      // per-node terms staged for a balanced node sum (else summed per wavenumber)
  double dT;
  const double* is64;
  const double* ss64;
  const double* dhalf;
  const cd* gphase;
  int n0;            // index of this launch's first link
  const cd* Win;     // [3][K1] carried state w entering link n0, or null: w from U0
  cd* Wout;          // [3][K1] carried state w after the last link, or null
  unsigned* status;  // set to ARP_ETIMEOUT if a wait gives up (0 on entry), or null
  int skip_first;    // test hook: CTA 0 does not send its first partial sums, so the owners' waits give up
};

// mbarrier and asynchronous remote-store primitives (PTX, sm_90 and later).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cluster_addr(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase of `parity` to complete, at most kBarrierTimeoutNs; on
// giving up records ARP_ETIMEOUT and clears `alive` (later waits return at once).
__device__ __forceinline__ void mbar_wait(unsigned bar, unsigned parity, unsigned* status, bool& alive) {
  if (!alive || mbar_test(bar, parity)) return;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_test(bar, parity))
    if (globaltimer_ns() - t0 > kBarrierTimeoutNs) {
      if (status) atomicCAS(status, 0u, (unsigned)ARP_ETIMEOUT);
      alive = false;
      return;
    }
}
// (no memory clobber: the value travels in registers, and the volatile waits,
// which do clobber memory, keep every later read of a received buffer after them)
__device__ __forceinline__ void st_async(unsigned addr, cpx<float> v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar));
}
__device__ __forceinline__ void st_async(unsigned addr, cpx<double> v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "d"(v.x), "d"(v.y), "r"(bar));
}

template <int LOGN> struct ClusterBlock {
  static constexpr int value = (1 << LOGN) <= 256 ? 256 : 512;
};

// Shared memory: the two mbarriers (RED, WS; 16 bytes), FP64 per own wavenumber (w and e^{dT/2 D} gphase for 3
// branches, dhalf, the two eigen constants), the FFT lanes, twiddles,
// the node phases [q][3][K1] and weights, WS/ACC/EXCH and the eigen constants.
// The FP32 chain's transforms use the radix-16 plan at N = 1024 and 2048 (at
// N = 512 a state's 64 radix-16 butterflies leave it slower than radix 8).
template <typename T>
__host__ __device__ constexpr bool chain_r16(int logn) {
  return sizeof(T) == 4 && r16_available(logn) && logn >= 10;
}
template <typename T>
__host__ __device__ constexpr int chain_twiddles(int logn) {
  return chain_r16<T>(logn) ? twiddle16_count(logn) : twiddle_count(logn);
}

template <typename T>
inline size_t cluster_chain_smem_bytes(int logn, int q, int own, int C, bool ph_smem, bool tmp_smem) {
  const int K1 = ((1 << logn) - 1) / 3 + 1;
  return (size_t)16 + (size_t)6 * own * sizeof(cd) + (size_t)3 * own * sizeof(double) +
         (size_t)(2 * q * padded_len<T>(1 << logn) + chain_twiddles<T>(logn) + (ph_smem ? 3 * q * K1 : 0) + 3 * K1 +
                  (tmp_smem ? 3 * q * K1 : 0) + 3 * C * own) *
             sizeof(cpx<T>) +
         (size_t)(2 * K1 + q) * sizeof(T);
}

// Bytes CTA `rank` of a C-CTA cluster expects on its two mbarriers per time
// average: `red`, the partial sums of its own (branch, wavenumber) pairs from
// every rank (C x 3 x own pairs, own wavenumbers [min(K1, rank own),
// min(K1, rank own + own))); `ws`, the whole state (3 x K1 values) pushed by
// the owners.  elem_bytes = sizeof(cpx<T>) of the chain's precision.  The
// kernel arms its mbarriers with these counts; arp_chain_exchange_bytes
// returns them to the host.
struct ChainExchangeBytes {
  unsigned red, ws;
};
__host__ __device__ inline ChainExchangeBytes chain_exchange_bytes(int K1, int C, int rank, int own,
                                                                   int elem_bytes) {
  const int k0 = rank * own < K1 ? rank * own : K1;
  const int k1 = k0 + own < K1 ? k0 + own : K1;
  return {(unsigned)(C * 3 * (k1 - k0) * elem_bytes), (unsigned)(3 * K1 * elem_bytes)};
}

template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void chain_cluster_body(const ClusterChainArgs& a, const NbarTabs<T>& tb) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  constexpr int N = 1 << LOGN;
  constexpr int H = N / 2 + 1;
  constexpr int K = (N - 1) / 3;
  constexpr int K1 = K + 1;
  constexpr int PL = padded_len<T>(N);
  const int C = (int)cl.num_blocks();
  const int j = (int)cl.block_rank();
  const int q = a.q, own = a.own;
  const int m0 = min(a.M, j * q);
  const int nq = min(a.M, m0 + q) - m0;  // nodes of this CTA (may be 0)
  const int k0 = min(K1, j * own), k1 = min(K1, k0 + own);

  // Layout, each array aligned for its element: complex FP64 arrays first
  // (16-byte elements), then complex T arrays, then FP64 scalars, then T scalars.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned bar_red = smem_addr(smem_raw), bar_ws = bar_red + 8;  // mbarriers
  cd* W64 = reinterpret_cast<cd*>(smem_raw + 16);  // [3][own] FP64 w of the own wavenumbers
  cd* GPH = W64 + 3 * own;                    // [3][own] e^{dT/2 D} e^{-i omega dT/eps}
  cpx<T>* Z = reinterpret_cast<cpx<T>*>(GPH + 3 * own);
  cpx<T>* TW = Z + 2 * q * PL;
  constexpr bool R16 = chain_r16<T>(LOGN);
  cpx<T>* PHs = TW + chain_twiddles<T>(LOGN);  // [q][3][K1] phases of this CTA's nodes
  cpx<T>* WS = PHs + (a.ph_smem ? 3 * q * K1 : 0);  // [3][K1] state, written by the owners
  const cpx<T>* PH = a.ph_smem ? PHs : tb.avg.phase + (size_t)m0 * 3 * K1;
  cpx<T>* TMP = WS + 3 * K1;                  // [q][3][K1] weighted terms of this CTA's nodes
  cpx<T>* RED = TMP + (a.tmp_smem ? 3 * q * K1 : 0);  // [C][3][own] partial sums sent by each rank
  double* DH = reinterpret_cast<double*>(RED + 3 * C * own);  // [own] e^{-nu k^4 dT/2}
  double* IS64 = DH + own;                    // [own]
  double* SS64 = IS64 + own;                  // [own]
  T* IS = reinterpret_cast<T*>(SS64 + own);
  T* SS = IS + K1;
  T* WM = SS + K1;                            // [q] weights of this CTA's nodes

  {
    const cpx<T>* twg = R16 ? reinterpret_cast<const cpx<T>*>(tb.tw16) : tb.tw;
    for (int t = threadIdx.x; t < chain_twiddles<T>(LOGN); t += BLOCK) TW[t] = twg[t];
  }
  for (int k = threadIdx.x; k < K1; k += BLOCK) {
    IS[k] = tb.is[k];
    SS[k] = tb.ss[k];
  }
  if (a.ph_smem)
    for (int t = threadIdx.x; t < nq * 3 * K1; t += BLOCK) PHs[t] = tb.avg.phase[(size_t)m0 * 3 * K1 + t];
  for (int d = threadIdx.x; d < nq; d += BLOCK) WM[d] = tb.avg.weight[m0 + d];
  for (int k = k0 + (int)threadIdx.x; k < k1; k += BLOCK) {
    DH[k - k0] = a.dhalf[k];
    IS64[k - k0] = a.is64[k];
    SS64[k - k0] = a.ss64[k];
#pragma unroll
    for (int b = 0; b < 3; ++b) GPH[b * own + (k - k0)] = a.dhalf[k] * a.gphase[b * K1 + k];
  }
  // w = e^{dT/2 D} R^H U_0 (or the carried w of an earlier launch) for the own
  // wavenumbers; its float copy into every CTA's WS
  for (int k = k0 + (int)threadIdx.x; k < k1; k += BLOCK) {
    if (a.Win) {
#pragma unroll
      for (int b = 0; b < 3; ++b) W64[b * own + (k - k0)] = a.Win[b * K1 + k];
      continue;
    }
    cd x[3], e[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      x[f] = a.U0[f * H + k];
      if (k == 0) x[f].y = 0.0;
    }
    phys_to_eigen<double>(x, a.is64[k], a.ss64[k], e);
#pragma unroll
    for (int b = 0; b < 3; ++b) W64[b * own + (k - k0)] = a.dhalf[k] * e[b];
  }
  // owner thread t < 3 no: branch b and own wavenumber r; it keeps VT of the
  // next two links for its pair in registers
  const int no = k1 - k0;
  const bool owner_t = (int)threadIdx.x < 3 * no;
  const int ob = owner_t ? (int)threadIdx.x / no : 0;
  const int orr = owner_t ? (int)threadIdx.x - ob * no : 0;
  const int ok = k0 + orr;
  auto load_vt = [&](int n) {
    return (a.VT && owner_t && n < a.S) ? a.VT[((size_t)(a.n0 + n) * 3 + ob) * K1 + ok] : cd{0.0, 0.0};
  };
  cd vt_cur = load_vt(0), vt_nxt = load_vt(1);
  // bytes per time average: the C ranks' partial sums of the own pairs, and the whole state
  const ChainExchangeBytes xb = chain_exchange_bytes(K1, C, j, own, (int)sizeof(cpx<T>));
  const unsigned red_bytes = xb.red;
  const unsigned ws_bytes = xb.ws;
  if (threadIdx.x == 0) {
    mbar_init(bar_red, 1);
    mbar_init(bar_ws, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (no > 0) mbar_expect(bar_red, red_bytes);
    mbar_expect(bar_ws, ws_bytes);
  }
  __syncthreads();  // W64
  for (int t = threadIdx.x; t < C * 3 * no; t += BLOCK) {
    const int c = t / (3 * no), r3 = t - c * 3 * no;
    const int b = r3 / no, r = r3 - b * no;
    cl.map_shared_rank(WS, c)[b * K1 + k0 + r] = cvt<T>(W64[b * own + r]);
  }
  cl.sync();  // the initial state, and the initialised barriers, visible cluster-wide
  bool alive = true;
  bool stop = false;
  unsigned parity = 0;

#pragma unroll 1
  for (int n = 0; n < a.S && !stop; ++n) {
#pragma unroll 1
    for (int round = 0; round < 2; ++round, parity ^= 1u) {
      const bool last = n == a.S - 1 && round == 1;
      // 1: this CTA's nodes, all at once
      constexpr int ZE1 = zero_end<N>() + 1;
      for (int item = threadIdx.x; item < nq * ZE1; item += BLOCK) {
        const int d = item / ZE1, k = item - d * ZE1;
        cpx<T>* Z0 = Z + 2 * d * PL;
        if (k > K) {
          zero_mode<T, N, R16>(Z0, Z0 + PL, k);
          continue;
        }
        cpx<T> x[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) x[b] = PH[(d * 3 + b) * K1 + k] * WS[b * K1 + k];
        pack_mode<T, N, R16>(Z0, Z0 + PL, k, x, IS[k], SS[k]);
      }
      if (__syncthreads_or(!alive)) {  // a wait of this CTA gave up
        stop = true;
        break;
      }
      if constexpr (R16) {
        if (nq > 0) nonlinear_transform16<LOGN, BLOCK>(reinterpret_cast<cf*>(Z), reinterpret_cast<const cf*>(TW), nq);
      } else {
        if (nq > 0) nonlinear_transform<T, LOGN, BLOCK>(Z, nq, TW);
      }
      if (a.tmp_smem) {
        // weighted, back-rotated term of each (node, wavenumber)
        for (int item = threadIdx.x; item < nq * K1; item += BLOCK) {
          const int d = item / K1, k = item - d * K1;
          cpx<T> bn[3];
          const cpx<T>* Z0 = Z + 2 * d * PL;
          unpack_mode<T, N, R16>(Z0, Z0 + PL, k, IS[k], SS[k], bn);
#pragma unroll
          for (int b = 0; b < 3; ++b) TMP[(d * 3 + b) * K1 + k] = WM[d] * (conj(PH[(d * 3 + b) * K1 + k]) * bn[b]);
        }
        __syncthreads();
        // node sum in node order, stored into the owner's reduction buffer
        for (int i = threadIdx.x; i < 3 * K1; i += BLOCK) {
          cpx<T> s = mk<T>(0, 0);
          for (int d = 0; d < nq; ++d) s = s + TMP[d * 3 * K1 + i];
          const int b = i / K1, k = i - b * K1, owner = k / own;
          if (!(a.skip_first && j == 0 && n == 0 && round == 0))
            st_async(cluster_addr(smem_addr(RED + (j * 3 + b) * own + (k - owner * own)), owner), s,
                     cluster_addr(bar_red, owner));
        }
      } else {
        // the same sum, one thread per wavenumber over the nodes in order
        for (int k = threadIdx.x; k < K1; k += BLOCK) {
          cpx<T> s[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
          for (int d = 0; d < nq; ++d) {
            cpx<T> bn[3];
            const cpx<T>* Z0 = Z + 2 * d * PL;
            unpack_mode<T, N, R16>(Z0, Z0 + PL, k, IS[k], SS[k], bn);
#pragma unroll
            for (int b = 0; b < 3; ++b) s[b] = s[b] + WM[d] * (conj(PH[(d * 3 + b) * K1 + k]) * bn[b]);
          }
          const int owner = k / own;
          const unsigned rbar = cluster_addr(bar_red, owner);
          if (!(a.skip_first && j == 0 && n == 0 && round == 0))
#pragma unroll
            for (int b = 0; b < 3; ++b)
              st_async(cluster_addr(smem_addr(RED + (j * 3 + b) * own + (k - owner * own)), owner), s[b], rbar);
        }
      }
      // 3: own (branch, wavenumber): sum over the ranks in rank order, FP64
      // epilogue, and the float copy of the result into every CTA's WS
      if (owner_t) {
        mbar_wait(bar_red, parity, a.status, alive);  // 2
        if (threadIdx.x == 0 && alive && !last) mbar_expect(bar_red, red_bytes);
        cpx<T> sr = mk<T>(0, 0);
        for (int c = 0; c < C; ++c) sr = sr + RED[(c * 3 + ob) * own + orr];
        const cd sum = cvt<double>(sr);
        const int i = ob * own + orr;
        cd v;
        if (round == 0) {  // midpoint state w + dT/2 k1
          v = W64[i] + (0.5 * a.dT) * sum;
        } else {  // g = e^{dT/2 D} e^{-(dT/eps) L} (w + dT k2); next w = e^{dT/2 D} g + VT_n
          const cd g = GPH[i] * (W64[i] + a.dT * sum);
          a.Ge[((size_t)(a.n0 + n) * 3 + ob) * K1 + ok] = g;
          v = DH[orr] * g + vt_cur;
          W64[i] = v;
          vt_cur = vt_nxt;
          vt_nxt = load_vt(n + 2);
        }
        if (!last) {
          const cpx<T> vt = cvt<T>(v);
          const unsigned ws = smem_addr(WS + ob * K1 + ok);
          for (int c = 0; c < C; ++c) st_async(cluster_addr(ws, c), vt, cluster_addr(bar_ws, c));
        }
      }
      if (!last) {
        mbar_wait(bar_ws, parity, a.status, alive);  // 4
        if (threadIdx.x == 0 && alive) mbar_expect(bar_ws, ws_bytes);
      }
    }
  }
  if (__syncthreads_or(!alive)) {
    // a wait gave up: leave stores of other CTAs still in flight a bounded moment to land
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 100000ull) {
    }
  }
  if (a.Wout)
    for (int k = k0 + (int)threadIdx.x; k < k1; k += BLOCK) {
#pragma unroll
      for (int b = 0; b < 3; ++b) a.Wout[b * K1 + k] = W64[b * own + (k - k0)];
    }
  cl.sync();  // no CTA leaves while another may still store into its shared memory
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) chain_cluster_kernel(ClusterChainArgs a, NbarTabs<T> tb) {
  chain_cluster_body<T, LOGN, BLOCK>(a, tb);
}

// Shared-memory plan of the cluster chain for one instance with C CTAs: stage
// what fits, the node phases before the per-node terms.  The phases are read
// at every time average and otherwise come from global memory, which a CTA's
// lanes leave too little L1 to cache (N = 1024, M = 128: the chain with them
// staged and the node sum one thread per wavenumber takes 14.7 ms against
// 17.8 ms with the terms staged instead).
struct ClusterPlan {
  int q, own, ph_smem, tmp_smem;
  size_t smem;  // > kMaxSmem if it does not fit at all
};
constexpr size_t kMaxSmem = 227 * 1024;

template <typename T>
inline ClusterPlan cluster_plan(int logn, int M, int K1, int C) {
  ClusterPlan p{(M + C - 1) / C, (K1 + C - 1) / C, 1, 1, 0};
  p.smem = cluster_chain_smem_bytes<T>(logn, p.q, p.own, C, true, true);
  if (p.smem > kMaxSmem) {
    p.tmp_smem = 0;
    p.smem = cluster_chain_smem_bytes<T>(logn, p.q, p.own, C, true, false);
  }
  if (p.smem > kMaxSmem) {
    p.ph_smem = 0;
    p.tmp_smem = 1;
    p.smem = cluster_chain_smem_bytes<T>(logn, p.q, p.own, C, false, true);
  }
  if (p.smem > kMaxSmem) {
    p.tmp_smem = 0;
    p.smem = cluster_chain_smem_bytes<T>(logn, p.q, p.own, C, false, false);
  }
  return p;
}

// Launch configuration of `count` clusters of C CTAs of `kern`; true if at
// least one such cluster can be resident (not queried when `known_fit`: the
// caller has checked this size on the current context's SMs before).
inline bool cluster_config(const void* kern, int C, int block, size_t smem, int count, cudaStream_t s,
                           cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, bool known_fit = false) {
  if (smem > kMaxSmem) return false;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *cfg = cudaLaunchConfig_t{};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->gridDim = dim3(C * count);
  cfg->blockDim = dim3(block);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = s;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  if (known_fit) return true;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, kern, cfg);
  if (e != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Launches the cluster chain (g_n into Ge; U and the G cache follow from
// finish_body); ARP_EINVAL (nothing launched) if no cluster of 16 or 8 CTAs
// with this kernel's shared memory can be scheduled.
template <typename T, int LOGN>
arp_status launch_cluster_chain_n(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                  const ChainRange* rg) {
  constexpr int BLOCK = ClusterBlock<LOGN>::value;
  const void* kern = (const void*)chain_cluster_kernel<T, LOGN, BLOCK>;
  for (int C : {16, 8}) {
    if (rg && rg->cluster && rg->cluster != C) continue;
    const ClusterPlan p = cluster_plan<T>(LOGN, c->M, c->K1, C);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const bool known = rg && rg->cluster == C && !rg->check_only;
    if (!cluster_config(kern, C, BLOCK, p.smem, 1, s, &cfg, attr, known)) continue;
    if (rg && rg->check_only) return ARP_OK;
    ClusterChainArgs a{VT, U0, Ge, rg ? rg->nl : c->slices, c->M, p.q, p.own, p.ph_smem, p.tmp_smem, c->dT,
                       c->inv_sig64, c->sk_sig64, c->dhalf, c->gphase, rg ? rg->n0 : 0, rg ? rg->Win : nullptr,
                       rg ? rg->Wout : nullptr, c->sync + 1, c->skip_arrival == 2};
    if (c->skip_arrival == 2) c->skip_arrival = 0;  // one launch
    NbarTabs<T> tb = nbar_tabs<T>(c);
    void* args[] = {&a, &tb};
    return check_cuda(c, cudaLaunchKernelExC(&cfg, kern, args), "cluster chain: launch");
  }
  return fail(c, ARP_EINVAL, "cluster chain: no cluster of 16 or 8 blocks fits");
}

template <typename T>
arp_status launch_cluster_chain_prec(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                     const ChainRange* rg) {
  switch (c->logN) {
    case 3: return launch_cluster_chain_n<T, 3>(c, U0, Ge, VT, s, rg);
    case 4: return launch_cluster_chain_n<T, 4>(c, U0, Ge, VT, s, rg);
    case 5: return launch_cluster_chain_n<T, 5>(c, U0, Ge, VT, s, rg);
    case 6: return launch_cluster_chain_n<T, 6>(c, U0, Ge, VT, s, rg);
    case 7: return launch_cluster_chain_n<T, 7>(c, U0, Ge, VT, s, rg);
    case 8: return launch_cluster_chain_n<T, 8>(c, U0, Ge, VT, s, rg);
    case 9: return launch_cluster_chain_n<T, 9>(c, U0, Ge, VT, s, rg);
    case 10: return launch_cluster_chain_n<T, 10>(c, U0, Ge, VT, s, rg);
    case 11: return launch_cluster_chain_n<T, 11>(c, U0, Ge, VT, s, rg);
    default: return fail(c, ARP_EINVAL, "cluster chain: unsupported grid size");
  }
}

}  // namespace arp

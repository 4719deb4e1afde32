// tc_gemm.cuh -- split-precision GEMM on the 5th-generation tensor cores
// (sm_100 family: tcgen05.mma, accumulators in tensor memory, operands staged
// in shared memory by the tensor memory accelerator), written with inline PTX.
//
//   C (M x Ncol, FP32) = sum over products p of  A_{a(p)} . B_{b(p)}^T
//
// A (M x K) and B (Ncol x K) are both K-major (K contiguous) and are stored as
// `parts` stacked copies [part][rows][K] holding the high, (middle,) low parts
// of a split of FP32 data into the MMA's input type (TF32 or BF16).  The
// products accumulate in FP32 in tensor memory, one accumulator per product
// order (see the splits below), in a fixed order (k block, then product, then
// the MMA's k step); the epilogue adds the accumulators smallest first.
//
// One CTA of 128 threads computes one 128 x 128 tile of C:
//   thread 0        TMA producer: for each K block, waits for a free stage and
//                   loads every part of the A and B tiles (128 rows x 128
//                   bytes each, 128-byte swizzle) onto the stage's mbarrier;
//   thread 32       MMA issuer: waits for a full stage, issues the products'
//                   tcgen05.mma (M = 128, N = 128, K = 32 bytes per
//                   instruction), and commits the stage back to the producer;
//                   after the last block it commits the accumulator;
//   warp 0          allocates the accumulators' tensor-memory columns (128 per
//                   accumulator, rounded up to a power of two) first and frees
//                   them last;
//   all 4 warps     epilogue: warp w reads accumulator lanes 32w..32w+31 (one
//                   row of C per thread) with tcgen05.ld and stores them,
//                   either as is or (the inverse DFT) as the products of the
//                   nonlinearity, split again into the input type.
// Every mbarrier wait is bounded (about a second of globaltimer); a wait that
// gives up sets bit 0 of *status, the thread stops issuing work, the producer
// waits (bounded) for the copies it has in flight, and the CTA still frees its
// tensor memory before it returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace arp {
namespace tc {

constexpr int kBM = 128;       // rows of a tile (the MMA's M, one tensor-memory lane per row)
constexpr int kBN = 128;       // columns of a tile (the MMA's N, tensor-memory columns)
constexpr int kRowBytes = 128; // K bytes of a tile row (one 128-byte swizzle atom)
constexpr int kThreads = 128;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of parity `parity` of the mbarrier to complete; false
// (and bit 0 of *status set) if it has not after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned* status) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && now_ns() - t0 > kWaitLimitNs) {
      atomicOr(status, 1u);
      return false;
    }
  }
}

// Tiled TMA load of box (c0 = K elements, c1 = rows, c2 = part) into shared
// memory, completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, unsigned bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tensor-memory allocation of `ncols` columns (a power of two >= 32) by one
// whole warp; the base address is written to shared memory at `slot`.
__device__ __forceinline__ void tmem_alloc(unsigned slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes
// with the 128-byte swizzle (8-row groups 1024 bytes apart): start address,
// leading offset unused (1), stride offset 1024 B, descriptor version 1,
// layout 2 = 128-byte swizzle.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: D in FP32, A and B of type `fmt` (kind::f16: 1 =
// BF16; kind::tf32: 2 = TF32), both K-major, N = kBN, M = kBM.
__host__ __device__ constexpr unsigned instr_desc(unsigned fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(kBN >> 3) << 17) | ((unsigned)(kBM >> 4) << 24);
}

template <int KIND>  // 0: kind::tf32, 1: kind::f16 (BF16 operands)
__device__ __forceinline__ void mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                    unsigned accumulate) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}
// The mbarrier at `bar` receives one arrival once every MMA this thread has
// issued so far has completed.
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's accumulator lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------------------
// Splits of FP32 values into the MMA input type.  x ~ sum of the parts; each
// part is the input-type rounding of what the earlier parts leave.

// Each split's products are ordered by their order (the sum of the two parts'
// indices, hence their size); products of one order accumulate in their own
// tensor-memory accumulator (acc(p) = the order), and the epilogue adds the
// accumulators smallest first, so the small correction terms are not rounded
// against the large running sum of the leading product at every MMA.

struct SplitTF32x3 {  // x = hi + lo, TF32 parts (cvt.rna); products hi.hi + hi.lo + lo.hi
  using E = float;
  static constexpr int kKind = 0, kFmt = 2, kParts = 2, kProducts = 3, kStages = 3, kAccs = 2;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  __host__ __device__ static constexpr int pa(int p) { return p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
  __host__ __device__ static constexpr int acc(int p) { return pa(p) + pb(p); }
  __device__ static float tf32(float x) {
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
  }
  __device__ static void split(float x, E* dst, size_t part_stride) {
    const float hi = tf32(x);
    dst[0] = hi;
    dst[part_stride] = x - hi;
  }
  __device__ static void split_d(double x, E* dst, size_t part_stride) {
    const float hi = tf32((float)x);
    dst[0] = hi;
    dst[part_stride] = (float)(x - (double)hi);
  }
};

struct SplitBF16x2 {  // x = hi + lo, BF16 parts; all four products hi.hi + hi.lo + lo.hi + lo.lo
  using E = __nv_bfloat16;
  static constexpr int kKind = 1, kFmt = 1, kParts = 2, kProducts = 4, kStages = 3, kAccs = 3;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  __host__ __device__ static constexpr int pa(int p) { return p >> 1; }
  __host__ __device__ static constexpr int pb(int p) { return p & 1; }
  __host__ __device__ static constexpr int acc(int p) { return pa(p) + pb(p); }
  __device__ static void split(float x, E* dst, size_t part_stride) {
    const E hi = __float2bfloat16_rn(x);
    dst[0] = hi;
    dst[part_stride] = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
  __device__ static void split_d(double x, E* dst, size_t part_stride) {
    const E hi = __float2bfloat16_rn((float)x);
    dst[0] = hi;
    dst[part_stride] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
  }
};

struct SplitBF16x3 {  // x = hi + mid + lo, BF16 parts; the six products whose parts' orders sum to <= 2
  using E = __nv_bfloat16;
  static constexpr int kKind = 1, kFmt = 1, kParts = 3, kProducts = 6, kStages = 2, kAccs = 3;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __host__ __device__ static constexpr int pa(int p) { return p == 2 ? 1 : (p == 4 ? 1 : (p == 5 ? 2 : 0)); }
  __host__ __device__ static constexpr int pb(int p) { return p == 1 ? 1 : (p == 3 ? 2 : (p == 4 ? 1 : 0)); }
  __host__ __device__ static constexpr int acc(int p) { return pa(p) + pb(p); }
  __device__ static void split(float x, E* dst, size_t part_stride) {
    const E hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(hi);
    const E mid = __float2bfloat16_rn(r1);
    dst[0] = hi;
    dst[part_stride] = mid;
    dst[2 * part_stride] = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  }
  __device__ static void split_d(double x, E* dst, size_t part_stride) {
    const E hi = __float2bfloat16_rn((float)x);
    const double r1 = x - (double)__bfloat162float(hi);
    const E mid = __float2bfloat16_rn((float)r1);
    dst[0] = hi;
    dst[part_stride] = mid;
    dst[2 * part_stride] = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(mid)));
  }
};

template <class S>
__host__ __device__ constexpr int stage_bytes() {
  return 2 * S::kParts * kBM * kRowBytes;  // A and B tiles of every part (kBN == kBM rows each)
}
template <class S>
__host__ __device__ constexpr size_t smem_bytes() {
  return (size_t)S::kStages * stage_bytes<S>() + 1024 /* alignment */ + 256 /* barriers, slot */;
}

// Epilogue of the tile: 0 = store C (FP32, column-major with leading dimension
// ldc, rows < m_valid, columns < ncols); 1 = the inverse DFT's products: the
// tile's columns are column groups of 4 (v1, h, v1_x, v2_x at grid point =
// row), and the three products -v1 v1_x, -v1 v2_x, -h v1 of group g at point
// j are split into P[part][3g + f][j] (row length ldp; rows j < m_valid).
constexpr int kEpiStore = 0;
constexpr int kEpiProducts = 1;

struct Epilogue {
  float* C;
  void* P;
  long long ncols;       // valid columns of C (kEpiStore) or of the GEMM (4 per group, kEpiProducts)
  int ldc;
  int ldp;
  long long p_part_stride;  // elements between parts of P
  int m_valid;
  unsigned* status;
};

// Tensor-memory columns of the S::kAccs accumulators of kBN columns (a power of two).
template <class S>
__host__ __device__ constexpr unsigned tmem_cols() {
  return S::kAccs * kBN <= 128 ? 128u : (S::kAccs * kBN <= 256 ? 256u : 512u);
}
// The first product of each accumulator (it overwrites instead of adding).
template <class S>
__host__ __device__ constexpr bool first_of_acc(int p) {
  return p == 0 || S::acc(p) != S::acc(p - 1);
}

// The accumulator row segment [c, c + 16) of this thread, accumulators added
// smallest first.
template <class S>
__device__ __forceinline__ void load_sum16(unsigned trow, int c, float (&v)[16]) {
  tmem_ld16(trow + (unsigned)((S::kAccs - 1) * kBN + c), v);
#pragma unroll
  for (int a = S::kAccs - 2; a >= 0; --a) {
    float w[16];
    tmem_ld16(trow + (unsigned)(a * kBN + c), w);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = w[i] + v[i];
  }
}

template <class S, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int kblocks,
                      Epilogue ep) {
  using E = typename S::E;
  constexpr int ST = S::kStages, PARTS = S::kParts, TILE = kBM * kRowBytes;
  constexpr int KSTEPS = kRowBytes / 32;        // MMA k steps per tile row (32 bytes each)
  constexpr int KELEMS = kRowBytes / (int)sizeof(E);
  constexpr unsigned IDESC = instr_desc(S::kFmt);
  extern __shared__ unsigned char smem_raw[];
  const unsigned raw = smem_u32(smem_raw);
  const unsigned base = (raw + 1023u) & ~1023u;  // the 128-byte swizzle wants 1024-byte aligned tiles
  const unsigned tiles = base;
  const unsigned bars = base + ST * stage_bytes<S>();
  const unsigned full0 = bars, empty0 = bars + 8 * ST, done = bars + 16 * ST, slot = bars + 16 * ST + 8;
  unsigned* slot_ptr = reinterpret_cast<unsigned*>(smem_raw + (slot - raw));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.y * kBN;
  auto a_tile = [&](int s, int part) { return tiles + (unsigned)(s * stage_bytes<S>() + part * TILE); };
  auto b_tile = [&](int s, int part) { return tiles + (unsigned)(s * stage_bytes<S>() + (PARTS + part) * TILE); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(slot, tmem_cols<S>());
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tmem = *reinterpret_cast<volatile unsigned*>(slot_ptr);

  if (threadIdx.x == 0) {
    // producer
    int issued = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % ST;
      const unsigned ph = (unsigned)(kb / ST) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, ep.status)) break;
      mbar_arrive_expect_tx(full0 + 8 * s, (unsigned)stage_bytes<S>());
#pragma unroll
      for (int p = 0; p < PARTS; ++p) tma_load_3d(a_tile(s, p), &tmA, full0 + 8 * s, kb * KELEMS, m0, p);
#pragma unroll
      for (int p = 0; p < PARTS; ++p) tma_load_3d(b_tile(s, p), &tmB, full0 + 8 * s, kb * KELEMS, n0, p);
      ++issued;
    }
    if (issued < kblocks) {
      // gave up: wait (bounded) for the copies in flight on each stage's last phase
      for (int kb = issued - 1; kb >= 0 && kb >= issued - ST; --kb)
        mbar_wait(full0 + 8 * (kb % ST), (unsigned)(kb / ST) & 1u, ep.status);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % ST;
      if (!mbar_wait(full0 + 8 * s, (unsigned)(kb / ST) & 1u, ep.status)) break;
      fence_after();
#pragma unroll
      for (int p = 0; p < S::kProducts; ++p) {
        const unsigned long long da = smem_desc(a_tile(s, S::pa(p)));
        const unsigned long long db = smem_desc(b_tile(s, S::pb(p)));
#pragma unroll
        for (int k = 0; k < KSTEPS; ++k)
          mma<S::kKind>(tmem + (unsigned)(S::acc(p) * kBN), da + 2ull * k, db + 2ull * k, IDESC,
                        (kb | k) != 0 || !first_of_acc<S>(p) ? 1u : 0u);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();

  // epilogue: one accumulator row per thread
  const bool ok = mbar_wait(done, 0u, ep.status);
  __syncwarp();  // tcgen05.ld is warp-wide: reconverge after the wait
  fence_after();
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
  const int row = m0 + warp * 32 + lane;
  if constexpr (EPI == kEpiStore) {
#pragma unroll 1
    for (int c = 0; c < kBN; c += 16) {
      float v[16];
      load_sum16<S>(trow, c, v);
      if (ok && row < ep.m_valid) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const long long col = (long long)n0 + c + i;
          if (col < ep.ncols) ep.C[col * ep.ldc + row] = v[i];
        }
      }
    }
  } else {
    E* P = static_cast<E*>(ep.P);
#pragma unroll 1
    for (int c = 0; c < kBN; c += 16) {
      float v[16];
      load_sum16<S>(trow, c, v);
      if (ok && row < ep.m_valid) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const long long col = (long long)n0 + c + 4 * g;
          if (col >= ep.ncols) break;
          const float v1 = v[4 * g], h = v[4 * g + 1], v1x = v[4 * g + 2], v2x = v[4 * g + 3];
          const float prod[3] = {-v1 * v1x, -v1 * v2x, -h * v1};
          const long long grp = col >> 2;
#pragma unroll
          for (int f = 0; f < 3; ++f) S::split(prod[f], P + (3 * grp + f) * ep.ldp + row, (size_t)ep.p_part_stride);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_free(tmem, tmem_cols<S>());
  }
}

}  // namespace tc
}  // namespace arp

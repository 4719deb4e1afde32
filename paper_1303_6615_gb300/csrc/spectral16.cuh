// spectral16.cuh -- a radix-16 plan of the nonlinearity's transforms for the
// FP32 fine sweep at N = 512, 1024 and 2048 (the fourth schedule): the same
// evaluation of N(u) as nonlinear_transform (inverse DFT of the two packed
// lanes, products, forward DFT, the 2/3 rule), with radix-16 outer stages at
// spans N and N/16 and a middle stage of span 2^(log2 N mod 4) (2, 4 or 8)
// fused with the products: five shared-memory round trips per evaluation
// instead of seven at N = 1024.
//
// Lane layout: element i of a lane at i ^ ((i >> 4) & 15) (bits 0-3 XORed with
// bits 4-7).  Each half-warp access of the plan's stages (radix-16 at span N:
// 16 consecutive j; at span N/16: 4 groups of 4 consecutive j; the middle stage:
// 16 consecutive items of R points) then hits 16 different bank pairs.
//
// A radix-16 item is one lane's butterfly (16 complex values in registers);
// the middle stage's item holds both lanes at R positions.  The span-N inverse
// stage takes inputs q = 6..9 (bins 3N/8 .. 5N/8-1, zero by the 2/3 rule) as
// zero without reading them; the span-N forward stage skips the outputs no
// evaluation reads (q = 6..9 of the first lane, q >= 6 of the second).
#pragma once

#include "spectral.cuh"

namespace arp {

__host__ __device__ constexpr bool r16_available(int logn) { return logn >= 9 && logn <= 11; }
__host__ __device__ constexpr int r16_log_mid(int logn) { return logn % 4; }  // 1, 2, 3 for N = 512, 1024, 2048
// Twiddle table of the radix-16 stages: the span-2^logL table holds
// tw16[(q-1) L/16 + j] = e^{-2 pi i q j / L}, q = 1..15, j < L/16; larger spans first.
__host__ __device__ constexpr int twiddle16_offset(int logn, int logL) {
  int off = 0;
  for (int l = logn; l > logL; l -= 4) off += 15 * ((1 << l) / 16);
  return off;
}
__host__ __device__ constexpr int twiddle16_count(int logn) { return twiddle16_offset(logn, r16_log_mid(logn)); }

// DFT of 16 points with root w = e^{SIGN 2 pi i / 16}, in place, natural order:
// four DFTs of 4 over n1 (x[4 n1 + n2]), the twiddles w^{n2 k1}, four DFTs of 4
// over n2.  Inputs whose bit is set in ZERO are zero and not read.
template <int SIGN, unsigned ZERO = 0u>
__device__ __forceinline__ void dft16(cf x[16]) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r = 0.70710678118654752440f;
  constexpr float S = (float)SIGN;
  cf a[4][4];  // a[n2][k1]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    const bool z0 = (ZERO >> n2) & 1u, z1 = (ZERO >> (4 + n2)) & 1u, z2 = (ZERO >> (8 + n2)) & 1u,
               z3 = (ZERO >> (12 + n2)) & 1u;
    const cf x0 = z0 ? mk<float>(0.f, 0.f) : x[n2], x1 = z1 ? mk<float>(0.f, 0.f) : x[4 + n2];
    const cf x2 = z2 ? mk<float>(0.f, 0.f) : x[8 + n2], x3 = z3 ? mk<float>(0.f, 0.f) : x[12 + n2];
    // the sums and differences of a DFT of 4, dropping the terms that are zero
    // (packed adds: the inputs are loads or twiddle products ending in an FMA)
    const cf e0 = z2 ? x0 : (z0 ? x2 : bsum(x0, x2)), e1 = z2 ? x0 : (z0 ? mk<float>(-x2.x, -x2.y) : bdif(x0, x2));
    const cf o0 = z3 ? x1 : (z1 ? x3 : bsum(x1, x3));
    const cf od = z3 ? x1 : (z1 ? mk<float>(-x3.x, -x3.y) : bdif(x1, x3));
    const cf o1 = SIGN > 0 ? mul_i(od) : mul_mi(od);
    a[n2][0] = bsum(e0, o0);
    a[n2][2] = bdif(e0, o0);
    a[n2][1] = e1 + o1;
    a[n2][3] = e1 - o1;
  }
  // twiddles w^{n2 k1}: w^1, w^2, w^3 (n2 = 1), w^2, w^4, w^6 (n2 = 2), w^3, w^6, w^9 (n2 = 3)
  auto w1 = [&](cf v) { return mk<float>(c1 * v.x - S * s1 * v.y, S * s1 * v.x + c1 * v.y); };
  auto w2 = [&](cf v) { return mk<float>(r * (v.x - S * v.y), r * (S * v.x + v.y)); };
  auto w3 = [&](cf v) { return mk<float>(s1 * v.x - S * c1 * v.y, S * c1 * v.x + s1 * v.y); };
  auto w4 = [&](cf v) { return SIGN > 0 ? mul_i(v) : mul_mi(v); };
  auto w6 = [&](cf v) { return mk<float>(-r * (v.x + S * v.y), r * (S * v.x - v.y)); };
  auto w9 = [&](cf v) { return mk<float>(-c1 * v.x + S * s1 * v.y, -S * s1 * v.x - c1 * v.y); };
  a[1][1] = w1(a[1][1]);
  a[1][2] = w2(a[1][2]);
  a[1][3] = w3(a[1][3]);
  a[2][1] = w2(a[2][1]);
  a[2][2] = w4(a[2][2]);
  a[2][3] = w6(a[2][3]);
  a[3][1] = w3(a[3][1]);
  a[3][2] = w6(a[3][2]);
  a[3][3] = w9(a[3][3]);
  // DFTs of 4 over n2; a pair keeps scalar adds where an entry is a bare
  // product (w^2, w^6: their adds contract) or a swap (w^4)
  dft4<float, SIGN, true, true>(a[0][0], a[1][0], a[2][0], a[3][0]);
  dft4<float, SIGN, false, true>(a[0][1], a[1][1], a[2][1], a[3][1]);
  dft4<float, SIGN, false, false>(a[0][2], a[1][2], a[2][2], a[3][2]);
  dft4<float, SIGN, false, true>(a[0][3], a[1][3], a[2][3], a[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    x[k1] = a[0][k1];
    x[k1 + 4] = a[1][k1];
    x[k1 + 8] = a[2][k1];
    x[k1 + 12] = a[3][k1];
  }
}

// Positions pidx16(base + q E), q = 0..15, of one radix-16 butterfly whose
// base and offsets occupy disjoint bits (base = g 16E + j, j < E): pidx16 is
// linear over GF(2), so pidx16(base + q E) = pidx16(base) ^ pidx16(q E), the
// second term a constant; for E >= 16 the offset q E lies above bits 0-3 and
// only its swizzle term is XORed in, the offset itself being added.
template <int E>
__device__ __forceinline__ void butterfly16_positions(int base, int at[16]) {
  const int sb = pidx16(base);
#pragma unroll
  for (int q = 0; q < 16; ++q) at[q] = E >= 16 ? (sb ^ ((q * E >> 4) & 15)) + q * E : sb ^ pidx16(q * E);
}

// One outer radix-16 stage of span L = 2^LOGL on the two lanes of each of
// `nstates` states (state d's lane l at Z + (2d + l) N; the items of one state
// are 2 N/16 consecutive ones), one lane's butterfly per item: DIF (inverse, sign +):
// DFT then multiply by conj(tw); DIT (forward, sign -): multiply by tw, then
// DFT; tw[(q-1) L/16 + j] = e^{-2 pi i q j / L}.  PRUNE 1: inputs q = 6..9 are
// zero and not read; PRUNE 2: outputs q = 6..9 of lane 0 and q >= 6 of lane 1
// are not stored.  Items: lane-major (item = lane N/16 + butterfly), or
// GROUPED: warp w takes butterflies 16w .. 16w+15 of both lanes (one per
// half-warp), which at span N/16 are the points 256w .. 256w+255.
template <int N, int BLOCK, int SIGN, bool DIF, int LOGL, int PRUNE = 0, bool GROUPED = false>
__device__ __forceinline__ void radix16_stage(cf* Z, const cf* tw, int nstates = 1) {
  constexpr int NB = N / 16;
  constexpr int E = 1 << (LOGL - 4);
  static_assert(BLOCK % (2 * NB) == 0 && (2 * NB) % 32 == 0, "whole states per block, whole warps per state");
  for (int vitem = threadIdx.x; vitem < nstates * 2 * NB; vitem += BLOCK) {
    const int d = vitem / (2 * NB), item = vitem - d * 2 * NB;
    const int lane = GROUPED ? (item >> 4) & 1 : item / NB;
    const int bidx = GROUPED ? ((item >> 5) << 4) | (item & 15) : item - lane * NB;
    cf* Zl = Z + (2 * d + lane) * N;
    const int j = bidx & (E - 1);
    const int base = ((bidx >> (LOGL - 4)) << LOGL) + j;
    int at[16];
    butterfly16_positions<E>(base, at);
    cf x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (PRUNE == 1 && q >= 6 && q <= 9) continue;
      x[q] = Zl[at[q]];
    }
    if (!DIF && j) {
#pragma unroll
      for (int q = 1; q < 16; ++q) x[q] = x[q] * tw[(q - 1) * E + j];
    }
    if (PRUNE == 1)
      dft16<SIGN, 0x03C0u>(x);
    else
      dft16<SIGN>(x);
    if (DIF && j) {
#pragma unroll
      for (int q = 1; q < 16; ++q) x[q] = x[q] * conj(tw[(q - 1) * E + j]);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (PRUNE == 2 && q >= 6 && (lane == 1 || q <= 9)) continue;
      Zl[at[q]] = x[q];
    }
  }
}

// The middle stage (span R = 2^(log2 N mod 4) = N/256, twiddles 1) on both
// lanes of each state: last inverse DFT, products, first forward DFT on the
// same R positions.  Per state, the state's warp w (N/8 threads per state,
// taken in the order of the radix-16 stages' items) takes the items of points
// 256w .. 256w+255, the points its own GROUPED span-N/16 stages read and
// write, so only the warp synchronises around this stage.
template <int LOGN, int BLOCK>
__device__ __forceinline__ void middle16_stage(cf* Z, int nstates = 1) {
  constexpr int N = 1 << LOGN;
  constexpr int R = 1 << r16_log_mid(LOGN);
  constexpr int ST = N / 8;  // threads per state
  static_assert(BLOCK % ST == 0 && R == N / 256, "one warp per 256 points");
  for (int vt = threadIdx.x; vt < nstates * ST; vt += BLOCK) {
  const int d = vt / ST, tl = vt - d * ST;
  cf* Z0 = Z + 2 * d * N;
  cf* Z1 = Z0 + N;
  const int w = tl >> 5, t = tl & 31;
#pragma unroll
  for (int r = 0; r < 8 / R; ++r) {
    const int i = (256 / R) * w + t + 32 * r;
    // q < R <= 8 sets only bits below those of R i and below bit 4, so
    // pidx16(R i + q) = pidx16(R i) ^ q
    const int p0 = pidx16(R * i);
    cf a[8], b[8];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      a[q] = Z0[p0 ^ q];
      b[q] = Z1[p0 ^ q];
    }
    if constexpr (R == 8) {
      dft8<float, +1>(a);
      dft8<float, +1>(b);
    } else if constexpr (R == 4) {
      dft4<float, +1>(a[0], a[1], a[2], a[3]);
      dft4<float, +1>(b[0], b[1], b[2], b[3]);
    } else {
      const cf sa = bsum(a[0], a[1]), da = bdif(a[0], a[1]), sb = bsum(b[0], b[1]), db = bdif(b[0], b[1]);
      a[0] = sa; a[1] = da; b[0] = sb; b[1] = db;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) products(a[q], b[q]);
    // the products are bare products: the first forward level keeps scalar adds
    if constexpr (R == 8) {
      dft8<float, -1, false>(a);
      dft8<float, -1, false>(b);
    } else if constexpr (R == 4) {
      dft4<float, -1, false, false>(a[0], a[1], a[2], a[3]);
      dft4<float, -1, false, false>(b[0], b[1], b[2], b[3]);
    } else {
      const cf sa = a[0] + a[1], da = a[0] - a[1], sb = b[0] + b[1], db = b[0] - b[1];
      a[0] = sa; a[1] = da; b[0] = sb; b[1] = db;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Z0[p0 ^ q] = a[q];
      Z1[p0 ^ q] = b[q];
    }
  }
  }
}

// Inverse transform, products and forward transform of the two lanes of each
// of `nstates` states (state d's lanes at Z + 2dN and Z + (2d+1)N; entry and
// exit synchronised).  TW: the radix-16 twiddle tables.  BLOCK is a multiple
// of N/8: a thread takes the same states, and within a state the same warp's
// points, in the span-N/16 stages and the middle stage.
template <int LOGN, int BLOCK>
__device__ __forceinline__ void nonlinear_transform16(cf* Z, const cf* TW, int nstates = 1) {
  constexpr int N = 1 << LOGN;
  constexpr int MID = r16_log_mid(LOGN);
  static_assert(LOGN - 8 == MID, "two radix-16 stages and a middle stage");
  static_assert(BLOCK % (N / 8) == 0, "one radix-16 butterfly per thread and state");
  radix16_stage<N, BLOCK, +1, true, LOGN, 1>(Z, TW + twiddle16_offset(LOGN, LOGN), nstates);
  __syncthreads();
  // span N/16, middle and span N/16 again touch each warp's own 256 points
  radix16_stage<N, BLOCK, +1, true, LOGN - 4, 0, true>(Z, TW + twiddle16_offset(LOGN, LOGN - 4), nstates);
  __syncwarp();
  middle16_stage<LOGN, BLOCK>(Z, nstates);
  __syncwarp();
  radix16_stage<N, BLOCK, -1, false, LOGN - 4, 0, true>(Z, TW + twiddle16_offset(LOGN, LOGN - 4), nstates);
  __syncthreads();
  radix16_stage<N, BLOCK, -1, false, LOGN, 2>(Z, TW + twiddle16_offset(LOGN, LOGN), nstates);
  __syncthreads();
}

}  // namespace arp

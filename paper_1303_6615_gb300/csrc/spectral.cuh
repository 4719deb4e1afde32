// spectral.cuh -- block-cooperative evaluation of the RSW nonlinearity
// N(u) = -(v1 v1_x, v1 v2_x, (h v1)_x) in L's eigen coordinates (Sec. 6.1),
// pseudo-spectrally with the 2/3 rule, on one state held in shared memory.
//
// Data flow of one evaluation (per state, N grid points, K = (N-1)/3):
//   pack    per wavenumber k <= K: u_k = R_k a_k, then two complex spectra
//           Z0 = v1 + i h and Z1 = v1_x + i v2_x (each lane carries two real
//           fields of like magnitude, so neither inherits the other's rounding
//           error; negative k by Hermitian symmetry); zero above K.
//   inverse length-N complex DFT (sign +) of Z0 and Z1 as in-place radix-8
//           decimation-in-frequency stages: natural-order spectrum in,
//           physical samples out in digit-reversed order.
//   product pointwise (order does not matter): Z0 <- (-v1 v1_x) + i(-v1 v2_x),
//           Z1 <- (-h v1) + i 0 (the products of like magnitude share a lane); fused with the last inverse and the first
//           forward stage, whose butterflies touch the same positions.
//   forward length-N complex DFT (sign -) as in-place decimation-in-time
//           stages in the mirrored order: digit-reversed samples in, natural
//           spectrum out.
// The stage spans are N, N/8, ... down to a middle span of 8, 4 or 2 (the
// remainder of log2 N by 3); each outer stage is one shared-memory round trip
// of radix-8 butterflies held in registers.  Lane arrays are laid out so that
// the stages' accesses avoid bank conflicts (FP32 lanes of 128 points or more
// XOR-swizzled, the others padded with one slot every 16 float or 8 double
// elements; see pidx), and each outer stage reads its twiddles W_L^{qj},
// q = 1..7, from its own table laid out q-major (consecutive j).  The span-N
// stages skip the bins 3N/8 .. 5N/8-1, which the 2/3 rule keeps zero.
//   unpack  per k <= K: P1 = (Z0_k + conj Z0_{-k})/2, P2 = (Z0_k - conj Z0_{-k})/(2i),
//           P3 = Z1_k; N_k = (P1, P2, i k P3)/N; b_k = R_k^H N_k.
//
// R_k holds the closed-form orthonormal eigenvectors of L_k (Sec. 6.1):
//   r^0 = (0, i s k, 1)/sigma,  r^{+-} = (1, -+ i/sigma, +- s k/sigma)/sqrt 2,
//   s = F^-1/2, sigma = sqrt(1 + s^2 k^2), L_k r^alpha = i alpha sigma r^alpha.
#pragma once

#include "common.cuh"

namespace arp {

template <typename T> struct Consts;
template <> struct Consts<double> { static __device__ __forceinline__ double rsqrt2() { return 0.70710678118654752440; } };
template <> struct Consts<float> { static __device__ __forceinline__ float rsqrt2() { return 0.70710678118654752440f; } };

// u = R a: (v1, v2, h) from the branch amplitudes (a_-, a_0, a_+).
template <typename T>
__device__ __forceinline__ void eigen_to_phys(const cpx<T> a[3], T is, T ss, cpx<T> u[3]) {
  const T r2 = Consts<T>::rsqrt2();
  cpx<T> s = r2 * (a[2] + a[0]);
  cpx<T> d = r2 * (a[2] - a[0]);
  u[0] = s;
  u[1] = mul_i(ss * a[1] - is * d);
  u[2] = is * a[1] + ss * d;
}

// a = R^H u.
template <typename T>
__device__ __forceinline__ void phys_to_eigen(const cpx<T> u[3], T is, T ss, cpx<T> a[3]) {
  const T r2 = Consts<T>::rsqrt2();
  cpx<T> iv2 = mul_i(is * u[1]);  // i v2 / sigma
  cpx<T> hs = ss * u[2];          // s k h / sigma
  a[1] = is * u[2] - mul_i(ss * u[1]);
  a[2] = r2 * (u[0] + iv2 + hs);
  a[0] = r2 * (u[0] - iv2 - hs);
}

// Position of element i in a lane array of N points.  FP32 lanes of N >= 128
// points are not padded but XOR-swizzled inside each aligned 16-element block:
// bits 0-3 of i are XORed with S(bits 4-6 of i), S linear over GF(2) with bit
// 4 -> 0011, bit 5 -> 0110, bit 6 -> 1001.  Each half-warp access of the
// radix-8 stages varies four address bits: bits 0-3 for spans >= 128, bits
// {0,1,2,6}, {0,1,5,6} or {0,4,5,6} for spans 64, 32, 16; the middle stage
// varies {3,4,5,6}, {2,3,4,5} or {1,2,3,4}; for every such set the swizzled
// bits 0-3 are an invertible function of the varying bits, so the 16 threads
// hit 16 different bank pairs.  Other lanes (FP64, and FP32 below 128 points,
// where lanes of several states share a warp) keep one padding slot every
// 2^kShift elements.
template <typename T> struct Pad;
template <> struct Pad<float> { static constexpr int kShift = 4; };
template <> struct Pad<double> { static constexpr int kShift = 3; };
template <typename T>
__host__ __device__ constexpr bool swizzled_lanes(int n) {
  return sizeof(T) == 4 && n >= 128;
}
template <typename T, int N>
__host__ __device__ __forceinline__ constexpr int pidx(int i) {
  if constexpr (swizzled_lanes<T>(N)) {
    // S(b) for b = 0..7, one nibble each: 0, 3, 6, 5, 9, 10, 15, 12
    return i ^ (int)((0xCFA95630u >> (((unsigned)i >> 2) & 28u)) & 15u);
  } else {
    return i + (i >> Pad<T>::kShift);
  }
}
template <typename T>
__host__ __device__ constexpr int padded_len(int n) {
  return swizzled_lanes<T>(n) ? n : n + (n >> Pad<T>::kShift);
}

// Lane layout of the radix-16 plan (FP32, 512 <= N <= 2048, spectral16.cuh):
// element i at i ^ (bits 4-7 of i), no padding.
__host__ __device__ __forceinline__ constexpr int pidx16(int i) { return i ^ ((i >> 4) & 15); }

// Position of element i of an N-point lane: pidx, or pidx16 for the radix-16 plan's lanes.
template <typename T, int N, bool R16>
__host__ __device__ __forceinline__ constexpr int lane_pos(int i) {
  if constexpr (R16) return pidx16(i);
  else return pidx<T, N>(i);
}

// S(bits 4-6 of i): the swizzle term of pidx for swizzled lanes.
__host__ __device__ __forceinline__ constexpr int swz_term(int i) {
  return (int)((0xCFA95630u >> (((unsigned)i >> 2) & 28u)) & 15u);
}

// Positions pidx(base + q e), q = 0..7, of one radix-8 butterfly whose base
// and offsets occupy disjoint bits (base = g 8e + j with j < e, e a power of
// two): bits 4-6 of base + q e are then those of base XOR those of q e, and S
// is linear over GF(2), so the swizzle splits into S(base), computed once,
// and S(q e), a constant once e is known at compile time; for e >= 16 the
// offsets q e leave bits 0-3 alone and stay plain additions.  Equal to pidx
// term by term.
template <typename T, int N>
__device__ __forceinline__ void butterfly_positions(int base, int e, int at[8]) {
  if constexpr (swizzled_lanes<T>(N)) {
    const int sb = base ^ swz_term(base);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      at[q] = e >= 16 ? (sb ^ swz_term(q * e)) + q * e : (base + q * e) ^ swz_term(base) ^ swz_term(q * e);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) at[q] = pidx<T, N>(base + q * e);
  }
}

// Last wavenumber whose bins k and N-k must be zero before an inverse
// transform.  The first outer inverse stage (span N) reads bin j + q N/8 as its
// q-th input; the 2/3 rule leaves bins 3N/8 .. 5N/8-1 (q = 3, 4) zero, so that
// stage takes them as zero without reading them, and only K < k <= 3N/8 (the
// partner N-k = 5N/8 is a q = 5 input) must be cleared.  Without outer stages
// (N = 8) every bin is read.
template <int N>
__host__ __device__ constexpr int zero_end() {
  return (N > 8) ? 3 * N / 8 : N / 2;
}

// Stage plan for N = 2^LOGN: middle span 2^kLogMid (8 if 3 | log2 N, else 2
// or 4), outer radix-8 stages at spans 2^logL, logL = LOGN, LOGN-3, ... > kLogMid.
__host__ __device__ constexpr int stage_log_mid(int logn) { return (logn % 3 == 0) ? 3 : logn % 3; }
// Offset of the twiddle table of the outer stage of span 2^logL (tables of the
// larger spans first; each holds 7 L/8 entries).
__host__ __device__ constexpr int twiddle_offset(int logn, int logL) {
  int off = 0;
  for (int l = logn; l > logL; l -= 3) off += 7 * ((1 << l) / 8);
  return off;
}
__host__ __device__ constexpr int twiddle_count(int logn) { return twiddle_offset(logn, stage_log_mid(logn)); }

// Writes the inverse-transform input of wavenumber k (0 <= k <= K) for the
// eigen amplitudes a: Z0 = v1 + i h, Z1 = v1_x + i v2_x at bins k and N-k
// (R16: in the radix-16 plan's lane layout; likewise for zero_mode and unpack_mode).
template <typename T, int N, bool R16 = false>
__device__ __forceinline__ void pack_mode(cpx<T>* Z0, cpx<T>* Z1, int k, const cpx<T> a[3], T is, T ss) {
  cpx<T> u[3];
  eigen_to_phys(a, is, ss, u);
  const T kk = (T)k;
  cpx<T> A = u[0];
  cpx<T> B = kk * mul_i(u[0]);   // i k v1
  cpx<T> C = kk * mul_i(u[1]);   // i k v2
  cpx<T> D = u[2];
  if (k == 0) {
    // real fields: the k = 0 coefficients are real (and derivatives vanish)
    Z0[0] = mk<T>(A.x, D.x);
    Z1[0] = mk<T>((T)0, (T)0);
  } else {
    Z0[lane_pos<T, N, R16>(k)] = A + mul_i(D);
    Z0[lane_pos<T, N, R16>(N - k)] = conj(A) + mul_i(conj(D));
    Z1[lane_pos<T, N, R16>(k)] = B + mul_i(C);
    Z1[lane_pos<T, N, R16>(N - k)] = conj(B) + mul_i(conj(C));
  }
}

// Zeroes bins k and N-k (K < k <= N/2).
template <typename T, int N, bool R16 = false>
__device__ __forceinline__ void zero_mode(cpx<T>* Z0, cpx<T>* Z1, int k) {
  const cpx<T> z = mk<T>(0, 0);
  Z0[lane_pos<T, N, R16>(k)] = z;
  Z1[lane_pos<T, N, R16>(k)] = z;
  Z0[lane_pos<T, N, R16>(N - k)] = z;
  Z1[lane_pos<T, N, R16>(N - k)] = z;
}

// Reads the forward-transform output at wavenumber k (0 <= k <= K) and returns
// the eigen amplitudes b = R^H N_k of the nonlinearity.
template <typename T, int N, bool R16 = false>
__device__ __forceinline__ void unpack_mode(const cpx<T>* Z0, const cpx<T>* Z1, int k, T is, T ss, cpx<T> b[3]) {
  const T inv_n = (T)1 / (T)N;
  cpx<T> n3[3];
  if (k == 0) {
    cpx<T> q = Z0[0];
    n3[0] = mk<T>(q.x * inv_n, 0);
    n3[1] = mk<T>(q.y * inv_n, 0);
    n3[2] = mk<T>(0, 0);
  } else {
    cpx<T> q = Z0[lane_pos<T, N, R16>(k)];
    cpx<T> qm = conj(Z0[lane_pos<T, N, R16>(N - k)]);
    cpx<T> r = Z1[lane_pos<T, N, R16>(k)];
    const T half_n = (T)0.5 * inv_n;
    n3[0] = half_n * (q + qm);
    n3[1] = half_n * mul_mi(q - qm);
    n3[2] = ((T)k * inv_n) * mul_i(r);
  }
  phys_to_eigen(n3, is, ss, b);
}

// Length-4 DFT with root e^{sign 2 pi i/4} = sign * i.  P02 / P13: the pair
// (x0, x2) / (x1, x3) may use the packed butterfly adds (bsum, bdif), i.e.
// neither of its entries is a bare product; the second level's operands are
// sums and always may.  A product by +-i swaps components and stays scalar.
template <typename T, int SIGN, bool P02 = true, bool P13 = true>
__device__ __forceinline__ void dft4(cpx<T>& x0, cpx<T>& x1, cpx<T>& x2, cpx<T>& x3) {
  const cpx<T> a0 = P02 ? bsum(x0, x2) : x0 + x2, a1 = P02 ? bdif(x0, x2) : x0 - x2;
  const cpx<T> a2 = P13 ? bsum(x1, x3) : x1 + x3, d = P13 ? bdif(x1, x3) : x1 - x3;
  const cpx<T> a3 = SIGN > 0 ? mul_i(d) : mul_mi(d);
  x0 = bsum(a0, a2);
  x2 = bdif(a0, a2);
  x1 = a1 + a3;
  x3 = a1 - a3;
}

// Length-8 DFT with root w = e^{sign 2 pi i/8}: two length-4 DFTs of the even
// and odd entries, combined with w^1 = (1 + sign i)/sqrt2, w^2 = sign i,
// w^3 = (-1 + sign i)/sqrt2.  PACK: the inputs are no bare products (see dft4);
// the combination's products by w^1, w^3 keep their scalar (contractible) adds.
template <typename T, int SIGN, bool PACK = true>
__device__ __forceinline__ void dft8(cpx<T> x[8]) {
  cpx<T> e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  cpx<T> o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<T, SIGN, PACK, PACK>(e0, e1, e2, e3);
  dft4<T, SIGN, PACK, PACK>(o0, o1, o2, o3);
  const T r = Consts<T>::rsqrt2();
  const cpx<T> t1 = SIGN > 0 ? r * (o1 + mul_i(o1)) : r * (o1 - mul_i(o1));
  const cpx<T> t2 = SIGN > 0 ? mul_i(o2) : mul_mi(o2);
  const cpx<T> t3 = SIGN > 0 ? r * (mul_i(o3) - o3) : r * (mk<T>(-o3.x, -o3.y) - mul_i(o3));
  x[0] = bsum(e0, o0);
  x[4] = bdif(e0, o0);
  x[1] = e1 + t1;
  x[5] = e1 - t1;
  x[2] = e2 + t2;
  x[6] = e2 - t2;
  x[3] = e3 + t3;
  x[7] = e3 - t3;
}

// dft8 with x[3] = x[4] = 0: the even half's a0 = a1 = x[0] and the odd half's
// a2 = x[7], a3 = -(sign i) x[7]; the rest as dft8 (the same roundings).
template <typename T, int SIGN>
__device__ __forceinline__ void dft8_in34zero(cpx<T> x[8]) {
  const cpx<T> ea2 = bsum(x[2], x[6]);
  const cpx<T> ea3 = SIGN > 0 ? mul_i(bdif(x[2], x[6])) : mul_mi(bdif(x[2], x[6]));
  const cpx<T> e0 = bsum(x[0], ea2), e2 = bdif(x[0], ea2), e1 = x[0] + ea3, e3 = x[0] - ea3;
  const cpx<T> oa0 = bsum(x[1], x[5]), oa1 = bdif(x[1], x[5]);
  const cpx<T> oa3 = SIGN > 0 ? mul_mi(x[7]) : mul_i(x[7]);
  const cpx<T> o0 = bsum(oa0, x[7]), o2 = bdif(oa0, x[7]), o1 = oa1 + oa3, o3 = oa1 - oa3;
  const T r = Consts<T>::rsqrt2();
  const cpx<T> t1 = SIGN > 0 ? r * (o1 + mul_i(o1)) : r * (o1 - mul_i(o1));
  const cpx<T> t2 = SIGN > 0 ? mul_i(o2) : mul_mi(o2);
  const cpx<T> t3 = SIGN > 0 ? r * (mul_i(o3) - o3) : r * (mk<T>(-o3.x, -o3.y) - mul_i(o3));
  x[0] = bsum(e0, o0);
  x[4] = bdif(e0, o0);
  x[1] = e1 + t1;
  x[5] = e1 - t1;
  x[2] = e2 + t2;
  x[6] = e2 - t2;
  x[3] = e3 + t3;
  x[7] = e3 - t3;
}

// One outer radix-8 stage on `nlanes` lanes stored back to back (lane l at
// Z + l * padded_len(N)), span L = 2^logL (L/8 butterflies per group).
// tw: this stage's table, tw[(q-1) L/8 + j] = e^{-2 pi i q j / L}.
// DIF (inverse, sign +): DFT then multiply by conj(tw); DIT (forward, sign -):
// multiply by tw then DFT.  PRUNE (span N only, see zero_end): 1 = inputs
// q = 3, 4 are zero and not read; 2 = outputs q = 3, 4 are never read and not
// stored (their arithmetic drops out).
template <typename T, int N, int BLOCK, int SIGN, bool DIF, int PRUNE = 0>
__device__ __forceinline__ void radix8_stage(cpx<T>* Z, int nlanes, const cpx<T>* tw, int logL) {
  constexpr int PL = padded_len<T>(N);
  constexpr int NB = N / 8;
  const int e = 1 << (logL - 3);
  for (int item = threadIdx.x; item < nlanes * NB; item += BLOCK) {
    const int lane = item / NB;
    const int bidx = item - lane * NB;
    cpx<T>* Zl = Z + lane * PL;
    const int j = bidx & (e - 1);
    const int base = ((bidx >> (logL - 3)) << logL) + j;
    int at[8];
    butterfly_positions<T, N>(base, e, at);
    cpx<T> x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (PRUNE == 1 && (q == 3 || q == 4)) continue;
      x[q] = Zl[at[q]];
    }
    if (!DIF && j) {
#pragma unroll
      for (int q = 1; q < 8; ++q) x[q] = x[q] * tw[(q - 1) * e + j];
    }
    if (PRUNE == 1)
      dft8_in34zero<T, SIGN>(x);
    else
      dft8<T, SIGN>(x);
    if (DIF && j) {
#pragma unroll
      for (int q = 1; q < 8; ++q) x[q] = x[q] * conj(tw[(q - 1) * e + j]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (PRUNE == 2 && (q == 3 || q == 4)) continue;
      Zl[at[q]] = x[q];
    }
  }
}

// radix8_stage on both lanes of `npairs` lane pairs at once: one item is the
// butterfly at the same positions of lanes 2p and 2p+1, so the positions and
// twiddles are computed and loaded once for the two lanes and the thread runs
// two independent DFTs.  PRUNE 2 (last forward stage) also skips lane 2p+1's
// outputs q = 5..7: only its bins k <= K < 3N/8 are ever read (the third
// field's spectrum), while lane 2p needs bins k and N-k.  Arithmetic per lane
// as radix8_stage.
template <typename T, int N, int BLOCK, int SIGN, bool DIF, int PRUNE = 0>
__device__ __forceinline__ void radix8_stage_pairs(cpx<T>* Z, int npairs, const cpx<T>* tw, int logL) {
  constexpr int PL = padded_len<T>(N);
  constexpr int NB = N / 8;
  const int e = 1 << (logL - 3);
  for (int item = threadIdx.x; item < npairs * NB; item += BLOCK) {
    const int pair = item / NB;
    const int bidx = item - pair * NB;
    cpx<T>* Z0 = Z + 2 * pair * PL;
    cpx<T>* Z1 = Z0 + PL;
    const int j = bidx & (e - 1);
    const int base = ((bidx >> (logL - 3)) << logL) + j;
    int at[8];
    butterfly_positions<T, N>(base, e, at);
    cpx<T> x[8], y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (PRUNE == 1 && (q == 3 || q == 4)) continue;
      x[q] = Z0[at[q]];
      y[q] = Z1[at[q]];
    }
    if (!DIF && j) {
#pragma unroll
      for (int q = 1; q < 8; ++q) {
        const cpx<T> w = tw[(q - 1) * e + j];
        x[q] = x[q] * w;
        y[q] = y[q] * w;
      }
    }
    if (PRUNE == 1) {
      dft8_in34zero<T, SIGN>(x);
      dft8_in34zero<T, SIGN>(y);
    } else {
      dft8<T, SIGN>(x);
      dft8<T, SIGN>(y);
    }
    if (DIF && j) {
#pragma unroll
      for (int q = 1; q < 8; ++q) {
        const cpx<T> w = conj(tw[(q - 1) * e + j]);
        x[q] = x[q] * w;
        y[q] = y[q] * w;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (PRUNE == 2 && (q == 3 || q == 4)) continue;
      Z0[at[q]] = x[q];
      if (PRUNE == 2 && q > 4) continue;
      Z1[at[q]] = y[q];
    }
  }
}

// Products at one physical sample: z0 = v1 + i h, z1 = v1_x + i v2_x.
template <typename T>
__device__ __forceinline__ void products(cpx<T>& z0, cpx<T>& z1) {
  const T v1 = z0.x, h = z0.y, v1x = z1.x, v2x = z1.y;
  z0 = mk<T>(-v1 * v1x, -v1 * v2x);
  z1 = mk<T>(-h * v1, (T)0);
}

// The fused middle stage (span 2^LOGMID, twiddles all 1) on `npairs` lane
// pairs (lanes 2p and 2p+1 hold one state): last inverse DFT, products, first
// forward DFT, on the same positions.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void middle_stage(cpx<T>* Z, int npairs) {
  constexpr int N = 1 << LOGN;
  constexpr int PL = padded_len<T>(N);
  constexpr int LOGMID = stage_log_mid(LOGN);
  constexpr int R = 1 << LOGMID;
  for (int item = threadIdx.x; item < npairs * (N / R); item += BLOCK) {
    const int pair = item / (N / R);
    const int i = item - pair * (N / R);
    cpx<T>* Z0 = Z + 2 * pair * PL;
    cpx<T>* Z1 = Z0 + PL;
    // positions pidx(R i + q): R i and q < R <= 8 occupy disjoint bits below bit 4
    // for q, so the swizzle term is that of R i (XORing q in is adding it)
    int at[8];
#pragma unroll
    for (int q = 0; q < R; ++q)
      at[q] = swizzled_lanes<T>(N) ? ((R * i) ^ swz_term(R * i)) ^ q : pidx<T, N>(R * i + q);
    cpx<T> a[8], b[8];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      a[q] = Z0[at[q]];
      b[q] = Z1[at[q]];
    }
    if (R == 8) {
      dft8<T, +1>(a);
      dft8<T, +1>(b);
    } else if (R == 4) {
      dft4<T, +1>(a[0], a[1], a[2], a[3]);
      dft4<T, +1>(b[0], b[1], b[2], b[3]);
    } else {
      const cpx<T> s = bsum(a[0], a[1]), d = bdif(a[0], a[1]), t = bsum(b[0], b[1]), u = bdif(b[0], b[1]);
      a[0] = s; a[1] = d; b[0] = t; b[1] = u;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) products(a[q], b[q]);
    // the products are bare products: the first forward level keeps scalar adds
    if (R == 8) {
      dft8<T, -1, false>(a);
      dft8<T, -1, false>(b);
    } else if (R == 4) {
      dft4<T, -1, false, false>(a[0], a[1], a[2], a[3]);
      dft4<T, -1, false, false>(b[0], b[1], b[2], b[3]);
    } else {
      const cpx<T> s = a[0] + a[1], d = a[0] - a[1], t = b[0] + b[1], u = b[0] - b[1];
      a[0] = s; a[1] = d; b[0] = t; b[1] = u;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Z0[at[q]] = a[q];
      Z1[at[q]] = b[q];
    }
  }
}

// Inverse transform, products and forward transform of `nstates` states whose
// lane pairs are stored back to back from Z (entry and exit synchronised).
// TW: the outer stages' twiddle tables.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void nonlinear_transform(cpx<T>* Z, int nstates, const cpx<T>* TW) {
  constexpr int N = 1 << LOGN;
  constexpr int LOGMID = stage_log_mid(LOGN);
  if constexpr (LOGN > LOGMID) {
    // span N first: bins 3N/8 .. 5N/8-1 are zero by the 2/3 rule
    radix8_stage<T, N, BLOCK, +1, true, 1>(Z, 2 * nstates, TW + twiddle_offset(LOGN, LOGN), LOGN);
    __syncthreads();
  }
#pragma unroll
  for (int logL = LOGN - 3; logL > LOGMID; logL -= 3) {
    radix8_stage<T, N, BLOCK, +1, true>(Z, 2 * nstates, TW + twiddle_offset(LOGN, logL), logL);
    __syncthreads();
  }
  middle_stage<T, LOGN, BLOCK>(Z, nstates);
  __syncthreads();
#pragma unroll
  for (int logL = LOGMID + 3; logL < LOGN; logL += 3) {
    radix8_stage<T, N, BLOCK, -1, false>(Z, 2 * nstates, TW + twiddle_offset(LOGN, logL), logL);
    __syncthreads();
  }
  if constexpr (LOGN > LOGMID) {
    // span N last: bins 3N/8 .. 5N/8-1 lie above the kept modes and are not read
    radix8_stage<T, N, BLOCK, -1, false, 2>(Z, 2 * nstates, TW + twiddle_offset(LOGN, LOGN), LOGN);
    __syncthreads();
  }
}

// nonlinear_transform with both lanes of a state in one butterfly item
// (radix8_stage_pairs): N/8 items per outer stage instead of N/4.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void nonlinear_transform_pairs(cpx<T>* Z, int nstates, const cpx<T>* TW) {
  constexpr int N = 1 << LOGN;
  constexpr int LOGMID = stage_log_mid(LOGN);
  if constexpr (LOGN > LOGMID) {
    radix8_stage_pairs<T, N, BLOCK, +1, true, 1>(Z, nstates, TW + twiddle_offset(LOGN, LOGN), LOGN);
    __syncthreads();
  }
#pragma unroll
  for (int logL = LOGN - 3; logL > LOGMID; logL -= 3) {
    radix8_stage_pairs<T, N, BLOCK, +1, true>(Z, nstates, TW + twiddle_offset(LOGN, logL), logL);
    __syncthreads();
  }
  middle_stage<T, LOGN, BLOCK>(Z, nstates);
  __syncthreads();
#pragma unroll
  for (int logL = LOGMID + 3; logL < LOGN; logL += 3) {
    radix8_stage_pairs<T, N, BLOCK, -1, false>(Z, nstates, TW + twiddle_offset(LOGN, logL), logL);
    __syncthreads();
  }
  if constexpr (LOGN > LOGMID) {
    radix8_stage_pairs<T, N, BLOCK, -1, false, 2>(Z, nstates, TW + twiddle_offset(LOGN, LOGN), LOGN);
    __syncthreads();
  }
}

}  // namespace arp

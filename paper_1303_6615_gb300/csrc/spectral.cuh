// spectral.cuh -- block-cooperative evaluation of the RSW nonlinearity
// N(u) = -(v1 v1_x, v1 v2_x, (h v1)_x) in L's eigen coordinates (Sec. 6.1),
// pseudo-spectrally with the 2/3 rule, on one state held in shared memory.
//
// Data flow of one evaluation (per state, N grid points, K = (N-1)/3):
//   pack    per wavenumber k <= K: u_k = R_k a_k, then two complex spectra
//           Z0 = v1 + i h and Z1 = v1_x + i v2_x (each lane carries two real
//           fields of like magnitude, so neither inherits the other's rounding
//           error; negative k by Hermitian symmetry); zero above K.
//   inverse length-N complex DFT (sign +) of Z0 and Z1 as in-place radix-4/2
//           decimation-in-frequency stages: natural-order spectrum in,
//           physical samples out in digit-reversed order.
//   product pointwise (order does not matter): Z0 <- (-v1 v1_x) + i(-v1 v2_x),
//           Z1 <- (-h v1) + i 0 (the products of like magnitude share a lane); fused with the last inverse and the first
//           forward stage, whose butterflies touch the same positions.
//   forward length-N complex DFT (sign -) as in-place decimation-in-time
//           stages in the mirrored order: digit-reversed samples in, natural
//           spectrum out.
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

// Writes the inverse-transform input of wavenumber k (0 <= k <= K) for the
// eigen amplitudes a: Z0 = v1 + i h, Z1 = v1_x + i v2_x at bins k and N-k.
template <typename T, int N>
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
    Z0[k] = A + mul_i(D);
    Z0[N - k] = conj(A) + mul_i(conj(D));
    Z1[k] = B + mul_i(C);
    Z1[N - k] = conj(B) + mul_i(conj(C));
  }
}

// Zeroes bins k and N-k (K < k <= N/2).
template <typename T, int N>
__device__ __forceinline__ void zero_mode(cpx<T>* Z0, cpx<T>* Z1, int k) {
  const cpx<T> z = mk<T>(0, 0);
  Z0[k] = z;
  Z1[k] = z;
  Z0[N - k] = z;
  Z1[N - k] = z;
}

// Reads the forward-transform output at wavenumber k (0 <= k <= K) and returns
// the eigen amplitudes b = R^H N_k of the nonlinearity.
template <typename T, int N>
__device__ __forceinline__ void unpack_mode(const cpx<T>* Z0, const cpx<T>* Z1, int k, T is, T ss, cpx<T> b[3]) {
  const T inv_n = (T)1 / (T)N;
  cpx<T> n3[3];
  if (k == 0) {
    cpx<T> q = Z0[0];
    n3[0] = mk<T>(q.x * inv_n, 0);
    n3[1] = mk<T>(q.y * inv_n, 0);
    n3[2] = mk<T>(0, 0);
  } else {
    cpx<T> q = Z0[k];
    cpx<T> qm = conj(Z0[N - k]);
    cpx<T> r = Z1[k];
    const T half_n = (T)0.5 * inv_n;
    n3[0] = half_n * (q + qm);
    n3[1] = half_n * mul_mi(q - qm);
    n3[2] = ((T)k * inv_n) * mul_i(r);
  }
  phys_to_eigen(n3, is, ss, b);
}

// Twiddle W_N^t = e^{sign 2 pi i t / N} from the table tw[t] = e^{-2 pi i t/N}, t < N/2.
template <typename T, int N, int SIGN>
__device__ __forceinline__ cpx<T> twiddle(const cpx<T>* tw, int t) {
  cpx<T> w = (t < N / 2) ? tw[t] : mk<T>(-tw[t - N / 2].x, -tw[t - N / 2].y);
  return SIGN > 0 ? conj(w) : w;
}

// Length-4 DFT with root e^{sign 2 pi i/4} = sign * i.
template <typename T, int SIGN>
__device__ __forceinline__ void dft4(cpx<T>& x0, cpx<T>& x1, cpx<T>& x2, cpx<T>& x3) {
  cpx<T> a0 = x0 + x2, a1 = x0 - x2, a2 = x1 + x3;
  cpx<T> a3 = SIGN > 0 ? mul_i(x1 - x3) : mul_mi(x1 - x3);
  x0 = a0 + a2;
  x2 = a0 - a2;
  x1 = a1 + a3;
  x3 = a1 - a3;
}

// One radix-4 stage on both lanes, span L (L/4 butterflies per group).
// DIF: DFT then twiddle W_L^{qj}; DIT: twiddle then DFT.
template <typename T, int N, int BLOCK, int SIGN, bool DIF>
__device__ __forceinline__ void radix4_stage(cpx<T>* Z0, cpx<T>* Z1, const cpx<T>* tw, int logL) {
  const int quarter = 1 << (logL - 2);
  const int tstride = N >> logL;  // N / L
  constexpr int NB = N / 4;
  for (int item = threadIdx.x; item < 2 * NB; item += BLOCK) {
    cpx<T>* Z = (item < NB) ? Z0 : Z1;
    const int bidx = (item < NB) ? item : item - NB;
    const int j = bidx & (quarter - 1);
    const int base = ((bidx >> (logL - 2)) << logL) + j;
    cpx<T> x0 = Z[base], x1 = Z[base + quarter], x2 = Z[base + 2 * quarter], x3 = Z[base + 3 * quarter];
    const int t = j * tstride;
    if (DIF) {
      dft4<T, SIGN>(x0, x1, x2, x3);
      if (j) {
        x1 = x1 * twiddle<T, N, SIGN>(tw, t);
        x2 = x2 * twiddle<T, N, SIGN>(tw, 2 * t);
        x3 = x3 * twiddle<T, N, SIGN>(tw, 3 * t);
      }
    } else {
      if (j) {
        x1 = x1 * twiddle<T, N, SIGN>(tw, t);
        x2 = x2 * twiddle<T, N, SIGN>(tw, 2 * t);
        x3 = x3 * twiddle<T, N, SIGN>(tw, 3 * t);
      }
      dft4<T, SIGN>(x0, x1, x2, x3);
    }
    Z[base] = x0;
    Z[base + quarter] = x1;
    Z[base + 2 * quarter] = x2;
    Z[base + 3 * quarter] = x3;
  }
}

// Products at one physical sample: z0 = v1 + i h, z1 = v1_x + i v2_x.
template <typename T>
__device__ __forceinline__ void products(cpx<T>& z0, cpx<T>& z1) {
  const T v1 = z0.x, h = z0.y, v1x = z1.x, v2x = z1.y;
  z0 = mk<T>(-v1 * v1x, -v1 * v2x);
  z1 = mk<T>(-h * v1, (T)0);
}

// The fused middle stage: last inverse (DIF) stage, whose twiddles are all 1,
// the products, and the first forward (DIT) stage, which touches the same
// positions.  Span 2 when log2 N is odd, else 4.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void middle_stage(cpx<T>* Z0, cpx<T>* Z1) {
  constexpr int N = 1 << LOGN;
  if (LOGN & 1) {
    for (int i = threadIdx.x; i < N / 2; i += BLOCK) {
      cpx<T> a0 = Z0[2 * i], a1 = Z0[2 * i + 1];
      cpx<T> b0 = Z1[2 * i], b1 = Z1[2 * i + 1];
      cpx<T> s = a0 + a1, d = a0 - a1;
      cpx<T> t = b0 + b1, e = b0 - b1;
      products(s, t);
      products(d, e);
      Z0[2 * i] = s + d;
      Z0[2 * i + 1] = s - d;
      Z1[2 * i] = t + e;
      Z1[2 * i + 1] = t - e;
    }
  } else {
    for (int i = threadIdx.x; i < N / 4; i += BLOCK) {
      cpx<T> a0 = Z0[4 * i], a1 = Z0[4 * i + 1], a2 = Z0[4 * i + 2], a3 = Z0[4 * i + 3];
      cpx<T> b0 = Z1[4 * i], b1 = Z1[4 * i + 1], b2 = Z1[4 * i + 2], b3 = Z1[4 * i + 3];
      dft4<T, +1>(a0, a1, a2, a3);
      dft4<T, +1>(b0, b1, b2, b3);
      products(a0, b0);
      products(a1, b1);
      products(a2, b2);
      products(a3, b3);
      dft4<T, -1>(a0, a1, a2, a3);
      dft4<T, -1>(b0, b1, b2, b3);
      Z0[4 * i] = a0; Z0[4 * i + 1] = a1; Z0[4 * i + 2] = a2; Z0[4 * i + 3] = a3;
      Z1[4 * i] = b0; Z1[4 * i + 1] = b1; Z1[4 * i + 2] = b2; Z1[4 * i + 3] = b3;
    }
  }
}

// Span exponents of the outer stages: inverse stages run logL = LOGN, LOGN-2,
// ... > kLogMid; forward stages run logL = kLogMid+2, ..., LOGN.
template <int LOGN> struct StagePlan { static constexpr int kLogMid = (LOGN & 1) ? 1 : 2; };

// Inverse transform, products and forward transform of the lanes Z0, Z1
// (entry and exit synchronised).  tw: e^{-2 pi i t/N}, t < N/2.
template <typename T, int LOGN, int BLOCK>
__device__ __forceinline__ void nonlinear_transform(cpx<T>* Z0, cpx<T>* Z1, const cpx<T>* tw) {
  constexpr int N = 1 << LOGN;
  constexpr int LOGMID = StagePlan<LOGN>::kLogMid;
#pragma unroll 1
  for (int logL = LOGN; logL > LOGMID; logL -= 2) {
    radix4_stage<T, N, BLOCK, +1, true>(Z0, Z1, tw, logL);
    __syncthreads();
  }
  middle_stage<T, LOGN, BLOCK>(Z0, Z1);
  __syncthreads();
#pragma unroll 1
  for (int logL = LOGMID + 2; logL <= LOGN; logL += 2) {
    radix4_stage<T, N, BLOCK, -1, false>(Z0, Z1, tw, logL);
    __syncthreads();
  }
}

}  // namespace arp

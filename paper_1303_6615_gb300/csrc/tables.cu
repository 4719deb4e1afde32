// tables.cu -- per-context tables, computed on the device in FP64 and rounded
// for the FP32 path:
//   * eigenvector constants of L_k (Sec. 6.1);
//   * per-stage FFT twiddles e^{-2 pi i q j / L} of the radix-8 stages, and of
//     the radix-16 stages of the FP32 sweep's radix-16 plan;
//   * ETDRK4 coefficients (Cox & Matthews) per wavenumber and eigen-branch for
//     the linear symbol lambda = -i omega/eps - nu k^4 (omega = alpha sigma_k);
//   * time-average nodes' phases e^{-i omega s_m}, s_m = T0 m/M, and weights
//     w_m = rho(m/M)/M with rho = C e^{-1/(s(1-s))}, int rho = 1 (Sec. 2,
//     Algorithm 1); C comes from a 1024-point trapezoid rule, which is exact to
//     rounding for this flat-ended integrand;
//   * coarse-step factors e^{-nu k^4 dT/2} and e^{-i omega dT/eps} (Algorithm 2).
#include <cmath>

#include "context.h"
#include "spectral.cuh"
#include "spectral16.cuh"

namespace arp {
namespace {

__device__ __forceinline__ cd cexp_d(cd z) {
  double s, c;
  sincos(z.y, &s, &c);
  const double e = exp(z.x);
  return {e * c, e * s};
}

// e^z - 1 without cancellation for small |z|: (e^x - 1) cos y - 2 sin^2(y/2) + i e^x sin y.
__device__ __forceinline__ cd cexpm1_d(cd z) {
  double s, c, sh, ch;
  sincos(z.y, &s, &c);
  sincos(0.5 * z.y, &sh, &ch);
  const double em1 = expm1(z.x);
  return {em1 * c - 2.0 * sh * sh, (em1 + 1.0) * s};
}

__device__ __forceinline__ cd cdiv_d(cd a, cd b) {
  const double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// phi_1, phi_2, phi_3 of z (phi_j(z) = sum_n z^n/(n+j)!).  |z| < 1: Horner sum of
// the phi_3 series (25 terms) and the identities phi_j = 1/j! + z phi_{j+1};
// otherwise phi_1 = (e^z - 1)/z and the same identities solved upward.
__device__ void phi123_d(cd z, cd& p1, cd& p2, cd& p3) {
  const double az = hypot(z.x, z.y);
  if (az < 1.0) {
    double c = 1.0;
    for (int i = 2; i <= 27; ++i) c /= (double)i;  // 1/27!
    cd s = {c, 0.0};
    for (int n = 23; n >= 0; --n) {
      c *= (double)(n + 4);                         // 1/(n+3)!
      s = {s.x * z.x - s.y * z.y + c, s.x * z.y + s.y * z.x};
    }
    p3 = s;
    p2 = {0.5 + (z.x * p3.x - z.y * p3.y), z.x * p3.y + z.y * p3.x};
    p1 = {1.0 + (z.x * p2.x - z.y * p2.y), z.x * p2.y + z.y * p2.x};
  } else {
    p1 = cdiv_d(cexpm1_d(z), z);
    p2 = cdiv_d({p1.x - 1.0, p1.y}, z);
    p3 = cdiv_d({p2.x - 0.5, p2.y}, z);
  }
}

__global__ void eigen_consts_kernel(int K1, double s, double* is64, double* ss64, float* is32, float* ss32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K1) return;
  const double sk = s * (double)k;
  const double sig = sqrt(1.0 + sk * sk);
  is64[k] = 1.0 / sig;
  ss64[k] = sk / sig;
  is32[k] = (float)(1.0 / sig);
  ss32[k] = (float)(sk / sig);
}

// Per-stage FFT twiddle tables: for each outer stage of span L = 2^logL,
// entries [(q-1) L/8 + j] = e^{-2 pi i q j / L}, q = 1..7, j < L/8.
__global__ void twiddle_kernel(int logn, cd* tw64, cf* tw32) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= twiddle_count(logn)) return;
  int off = 0, logL = logn;
  while (t >= off + 7 * ((1 << logL) / 8)) {
    off += 7 * ((1 << logL) / 8);
    logL -= 3;
  }
  const int e = (1 << logL) / 8;
  const int q = (t - off) / e + 1, j = (t - off) % e;
  double s, c;
  sincospi(-2.0 * (double)(q * j) / (double)(1 << logL), &s, &c);
  tw64[t] = {c, s};
  tw32[t] = {(float)c, (float)s};
}

// The radix-16 plan's twiddles (FP32 sweep, 512 <= N <= 2048): for each outer
// stage of span L = 2^logL, entries [(q-1) L/16 + j] = e^{-2 pi i q j / L},
// q = 1..15, j < L/16.
__global__ void twiddle16_kernel(int logn, cf* tw16) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= twiddle16_count(logn)) return;
  int off = 0, logL = logn;
  while (t >= off + 15 * ((1 << logL) / 16)) {
    off += 15 * ((1 << logL) / 16);
    logL -= 4;
  }
  const int e = (1 << logL) / 16;
  const int q = (t - off) / e + 1, j = (t - off) % e;
  double s, c;
  sincospi(-2.0 * (double)(q * j) / (double)(1 << logL), &s, &c);
  tw16[t] = {(float)c, (float)s};
}

// omega of branch b (alpha = b - 1) at wavenumber k.
__device__ __forceinline__ double omega_of(int b, int k, double s) {
  const double sk = s * (double)k;
  return (double)(b - 1) * sqrt(1.0 + sk * sk);
}

// One thread per wavenumber: branches alpha = 0 and +1 computed, alpha = -1 is
// the conjugate of alpha = +1 (lambda_- = conj(lambda_+)), kept exact so that
// real k = 0 fields stay real.
__global__ void etd_kernel(int K1, double s, double inv_eps, double nu, double h, cd* etd64, cf* etd32,
                           cf* elo32, cf* etd32c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K1) return;
  const double k4 = (double)k * (double)k * (double)k * (double)k;
  for (int b = 1; b <= 2; ++b) {
    const double om = omega_of(b, k, s);
    const cd lam = {-nu * k4, -om * inv_eps};
    const cd z = {h * lam.x, h * lam.y};
    const cd zh = {0.5 * z.x, 0.5 * z.y};
    cd p1, p2, p3, q1, q2, q3;
    phi123_d(z, p1, p2, p3);
    phi123_d(zh, q1, q2, q3);
    cd v[6];
    v[0] = cexp_d(z);
    v[1] = cexp_d(zh);
    v[2] = {0.5 * h * q1.x, 0.5 * h * q1.y};
    v[3] = {h * (p1.x - 3.0 * p2.x + 4.0 * p3.x), h * (p1.y - 3.0 * p2.y + 4.0 * p3.y)};
    v[4] = {2.0 * h * (p2.x - 2.0 * p3.x), 2.0 * h * (p2.y - 2.0 * p3.y)};
    v[5] = {h * (4.0 * p3.x - p2.x), h * (4.0 * p3.y - p2.y)};
    for (int j = 0; j < 6; ++j) {
      const int idx = (j * 3 + b) * K1 + k;
      etd64[idx] = v[j];
      etd32[idx] = {(float)v[j].x, (float)v[j].y};
      if (b == 2) {
        const int idm = (j * 3 + 0) * K1 + k;
        etd64[idm] = {v[j].x, -v[j].y};
        etd32[idm] = {(float)v[j].x, -(float)v[j].y};
      }
    }
    // low parts of E for the FP32 path's float-pair propagation
    const cf eh = {(float)v[0].x, (float)v[0].y};
    const cf el = {(float)(v[0].x - (double)eh.x), (float)(v[0].y - (double)eh.y)};
    elo32[b * K1 + k] = el;
    if (b == 2) elo32[k] = {el.x, -el.y};
    // compact copy: alpha = +1 complex, alpha = 0 real (its imaginary parts are zero)
    if (etd32c) {
      const cf c7[7] = {etd32[(0 * 3 + b) * K1 + k], etd32[(1 * 3 + b) * K1 + k], etd32[(2 * 3 + b) * K1 + k],
                        etd32[(3 * 3 + b) * K1 + k], etd32[(4 * 3 + b) * K1 + k], etd32[(5 * 3 + b) * K1 + k], el};
      float* z = reinterpret_cast<float*>(etd32c + 7 * K1);
      for (int j = 0; j < 7; ++j) {
        if (b == 2) etd32c[j * K1 + k] = c7[j];
        else z[j * K1 + k] = c7[j].x;
      }
    }
  }
}

// One block of 256 threads: C = 1 / int_0^1 e^{-1/(s(1-s))} ds (1024-point
// trapezoid, fixed-order reduction), then w_m = C e^{-1/(s_m(1-s_m))}/M at s = m/M.
__global__ void weights_kernel(int M, double* w64, float* w32) {
  __shared__ double part[256];
  constexpr int NT = 1024;
  double acc = 0.0;
  for (int j = threadIdx.x + 1; j < NT; j += 256) {
    const double sj = (double)j / NT;
    acc += exp(-1.0 / (sj * (1.0 - sj)));
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  const double C = (double)NT / part[0];
  for (int m = threadIdx.x; m < M; m += 256) {
    const double sm = (double)m / (double)M;
    const double r = (m == 0) ? 0.0 : C * exp(-1.0 / (sm * (1.0 - sm)));
    w64[m] = r / (double)M;
    w32[m] = (float)(r / (double)M);
  }
}

// phase[m][b][k] = e^{-i omega s_m}, s_m = T0 m / M.
__global__ void phase_kernel(int M, int K1, double s, double T0, cd* ph64, cf* ph32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K1) return;
  // nodes strided over gridDim.y (at most 65535 rows of blocks), so any M works
  for (int m = blockIdx.y; m < M; m += gridDim.y) {
    const double sm = T0 * (double)m / (double)M;
    const double arg = omega_of(2, k, s) * sm;
    double sn, cs;
    sincos(arg, &sn, &cs);
    const size_t base = (size_t)m * 3 * K1;
    ph64[base + 2 * K1 + k] = {cs, -sn};
    ph64[base + 0 * K1 + k] = {cs, sn};
    ph64[base + 1 * K1 + k] = {1.0, 0.0};
    ph32[base + 2 * K1 + k] = {(float)cs, -(float)sn};
    ph32[base + 0 * K1 + k] = {(float)cs, (float)sn};
    ph32[base + 1 * K1 + k] = {1.0f, 0.0f};
  }
}

// dhalf[k] = e^{-nu k^4 dT/2}; gphase[b][k] = e^{-i omega dT/eps};
// sth[b][k] = e^{lambda dT/2} = dhalf[k] e^{-i omega dT/(2 eps)}.
__global__ void coarse_consts_kernel(int K1, double s, double nu, double dT, double inv_eps, double* dhalf, cd* gph,
                                     cd* sth) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K1) return;
  const double k4 = (double)k * (double)k * (double)k * (double)k;
  dhalf[k] = exp(-nu * k4 * 0.5 * dT);
  const double arg = omega_of(2, k, s) * dT * inv_eps;
  double sn, cs;
  sincos(arg, &sn, &cs);
  gph[2 * K1 + k] = {cs, -sn};
  gph[0 * K1 + k] = {cs, sn};
  gph[1 * K1 + k] = {1.0, 0.0};
  double sh, ch;
  sincos(0.5 * arg, &sh, &ch);
  const double d = dhalf[k];
  sth[2 * K1 + k] = {d * ch, -d * sh};
  sth[0 * K1 + k] = {d * ch, d * sh};
  sth[1 * K1 + k] = {d, 0.0};
}

}  // namespace

arp_status build_tables(arp_ctx* c, cudaStream_t st) {
  const double s = 1.0 / std::sqrt(c->F);
  const double inv_eps = std::isinf(c->eps) ? 0.0 : 1.0 / c->eps;
  const double T0 = c->T0_set ? c->T0 : c->dT * inv_eps;
  const int tb = 128;
  eigen_consts_kernel<<<(c->K1 + tb - 1) / tb, tb, 0, st>>>(c->K1, s, c->inv_sig64, c->sk_sig64, c->inv_sig32,
                                                           c->sk_sig32);
  twiddle_kernel<<<(c->N + tb - 1) / tb, tb, 0, st>>>(c->logN, c->tw64, c->tw32);
  // only a context's own allocation has the FP32 sweep's radix-16 table (the
  // allocation-free time average, which builds its tables in a static array, has none)
  if (r16_available(c->logN) && c->tw16_32)
    twiddle16_kernel<<<(c->N + tb - 1) / tb, tb, 0, st>>>(c->logN, c->tw16_32);
  etd_kernel<<<(c->K1 + tb - 1) / tb, tb, 0, st>>>(c->K1, s, inv_eps, c->nu, c->h, c->etd64, c->etd32, c->E_lo32,
                                                   c->etd32c);
  weights_kernel<<<1, 256, 0, st>>>(c->M, c->weight64, c->weight32);
  phase_kernel<<<dim3((c->K1 + tb - 1) / tb, c->M < 65535 ? c->M : 65535), tb, 0, st>>>(c->M, c->K1, s, T0, c->phase64, c->phase32);
  coarse_consts_kernel<<<(c->K1 + tb - 1) / tb, tb, 0, st>>>(c->K1, s, c->nu, c->dT, inv_eps, c->dhalf, c->gphase,
                                                               c->strang_h64);
  arp_status r = check_cuda(c, cudaGetLastError(), "table kernels");
  if (r != ARP_OK) return r;
  c->tables_dirty = false;
  return ARP_OK;
}

}  // namespace arp

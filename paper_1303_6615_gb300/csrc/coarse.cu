// coarse.cu -- FP64 glue of the asymptotic slow solver (Algorithm 2):
//   w = e^{dT/2 D} u; k1 = Nbar(w); k2 = Nbar(w + dT/2 k1); w = e^{dT/2 D}(w + dT k2);
//   G(u) = e^{-(dT/eps) L} w,
// and of the stand-alone time average (Algorithm 1).  Nbar itself runs in
// nbar_partial_kernel; here: the conversion to eigen coordinates, the
// fixed-order sum of the quadrature-chunk partials, and the epilogues.
#include "context.h"
#include "spectral.cuh"

namespace arp {
namespace {

// W[b][q][k] = (dhalf[k]) (R^H u[b])_q for k <= K; one thread per (b, k).
__global__ void to_eigen_kernel(const cd* __restrict__ u, cd* __restrict__ W, int batch, int H, int K1,
                                const double* __restrict__ is, const double* __restrict__ ss,
                                const double* __restrict__ dhalf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)batch * K1) return;
  const int b = (int)(t / K1), k = (int)(t % K1);
  const cd* src = u + (size_t)b * 3 * H;
  cd x[3], a[3];
  for (int f = 0; f < 3; ++f) {
    x[f] = src[f * H + k];
    if (k == 0) x[f].y = 0.0;
  }
  phys_to_eigen<double>(x, is[k], ss[k], a);
  const double d = dhalf ? dhalf[k] : 1.0;
  cd* dst = W + (size_t)b * 3 * K1;
  for (int q = 0; q < 3; ++q) dst[q * K1 + k] = d * a[q];
}

struct ReduceArgs {
  int mode, batch, H, K1, P;
  double dT;
  const cd* partial;
  const cd* W;
  cd* W2;
  cd* out;
  const cd* vadd;
  cd* out2;
  const double* is;
  const double* ss;
  const double* dhalf;
  const cd* gphase;
};

// One thread per (b, k), k < H: Nbar = sum_p partial[b][p] in chunk order, then
// the epilogue of the mode (see context.h).
__global__ void reduce_kernel(ReduceArgs r) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)r.batch * r.H) return;
  const int b = (int)(t / r.H), k = (int)(t % r.H);
  if (k >= r.K1) {
    if (r.mode != kReduceMid) {
      for (int f = 0; f < 3; ++f) {
        r.out[((size_t)b * 3 + f) * r.H + k] = {0.0, 0.0};
        if (r.out2) r.out2[((size_t)b * 3 + f) * r.H + k] = {0.0, 0.0};
      }
    }
    return;
  }
  cd nb[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
  const cd* src = r.partial + (size_t)b * r.P * 3 * r.K1;
  // chunk order; unrolled so that the loads of several chunks are in flight at once
#pragma unroll 8
  for (int p = 0; p < r.P; ++p)
    for (int q = 0; q < 3; ++q) nb[q] = nb[q] + src[((size_t)p * 3 + q) * r.K1 + k];
  const cd* w = r.W ? r.W + (size_t)b * 3 * r.K1 : nullptr;
  if (r.mode == kReduceMid) {
    for (int q = 0; q < 3; ++q)
      r.W2[((size_t)b * 3 + q) * r.K1 + k] = w[q * r.K1 + k] + (0.5 * r.dT) * nb[q];
    return;
  }
  cd g[3];
  if (r.mode == kReduceFinal) {
    for (int q = 0; q < 3; ++q)
      g[q] = r.dhalf[k] * (r.gphase[q * r.K1 + k] * (w[q * r.K1 + k] + r.dT * nb[q]));
  } else {
    for (int q = 0; q < 3; ++q) g[q] = nb[q];
  }
  cd u[3];
  eigen_to_phys<double>(g, r.is[k], r.ss[k], u);
  for (int f = 0; f < 3; ++f) {
    if (k == 0) u[f].y = 0.0;
    const size_t o = ((size_t)b * 3 + f) * r.H + k;
    r.out[o] = u[f];
    if (r.out2) r.out2[o] = r.vadd ? u[f] + r.vadd[o] : u[f];
  }
}

}  // namespace

arp_status launch_to_eigen(arp_ctx* c, const cd* u, cd* W, int batch, bool use_dhalf, cudaStream_t s) {
  const long long n = (long long)batch * c->K1;
  if (n == 0) return ARP_OK;
  to_eigen_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(u, W, batch, c->H, c->K1, c->inv_sig64, c->sk_sig64,
                                                              use_dhalf ? c->dhalf : nullptr);
  return check_cuda(c, cudaGetLastError(), "to_eigen: launch");
}

arp_status launch_nbar_reduce(arp_ctx* c, int mode, const cd* partial, const cd* W, cd* W2, cd* out_phys,
                              const cd* vadd, cd* out2_phys, int batch, cudaStream_t s) {
  const long long n = (long long)batch * c->H;
  if (n == 0) return ARP_OK;
  // the DFT-GEMM time average writes the whole node sum as one chunk
  ReduceArgs r{mode, batch, c->H, c->K1, dft_mode(c) ? 1 : c->P, c->dT, partial, W, W2, out_phys, vadd, out2_phys,
               c->inv_sig64, c->sk_sig64, c->dhalf, c->gphase};
  reduce_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(r);
  return check_cuda(c, cudaGetLastError(), "reduce: launch");
}

arp_status coarse_avg(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  for (int b0 = 0; b0 < batch; b0 += c->cchunk) {
    const int nb = batch - b0 < c->cchunk ? batch - b0 : c->cchunk;
    const size_t off = (size_t)b0 * 3 * c->H;
    arp_status r;
    if ((r = launch_to_eigen(c, in + off, c->W, nb, false, s)) != ARP_OK) return r;
    if ((r = launch_nbar_partial(c, c->W, c->partial, nb, s)) != ARP_OK) return r;
    if ((r = launch_nbar_reduce(c, kReduceAvg, c->partial, nullptr, nullptr, out + off, nullptr, nullptr, nb, s)) !=
        ARP_OK)
      return r;
  }
  return ARP_OK;
}

arp_status coarse_step(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  if (c->coarse_scheme == 1) return launch_strang_sweep(c, in, out, batch, true, s);
  for (int b0 = 0; b0 < batch; b0 += c->cchunk) {
    const int nb = batch - b0 < c->cchunk ? batch - b0 : c->cchunk;
    const size_t off = (size_t)b0 * 3 * c->H;
    arp_status r;
    if ((r = launch_to_eigen(c, in + off, c->W, nb, true, s)) != ARP_OK) return r;
    if ((r = launch_nbar_partial(c, c->W, c->partial, nb, s)) != ARP_OK) return r;
    if ((r = launch_nbar_reduce(c, kReduceMid, c->partial, c->W, c->W2, nullptr, nullptr, nullptr, nb, s)) != ARP_OK)
      return r;
    if ((r = launch_nbar_partial(c, c->W2, c->partial, nb, s)) != ARP_OK) return r;
    if ((r = launch_nbar_reduce(c, kReduceFinal, c->partial, c->W, nullptr, out + off, nullptr, nullptr, nb, s)) !=
        ARP_OK)
      return r;
  }
  return ARP_OK;
}

}  // namespace arp

// parareal.cu -- one iteration of the parareal method (Eq. 3.1, Algorithm 4):
//   U_0^k = u0,
//   U_{n+1}^k = G(U_n^k) + F(U_n^{k-1}) - G(U_n^{k-1}),   k >= 1,
// with the predictor U_{n+1}^0 = G(U_n^0).  F(U_n^{k-1}) for all slices runs
// as one batched fine sweep; V_n = F - G is formed in FP64 in parallel; the
// serial chain then evaluates G(U_n^k) slice after slice, keeping each value
// as G(U_n^{k-1}) for the next iteration; finally the stopping quantity
// max_n ||U_n^k - U_n^{k-1}|| / ||U_n^k|| (L2 over the three fields by
// Parseval: weight 1 at k = 0 and 2 above) is reduced in a fixed order.
#include <cmath>

#include "context.h"
#include "parareal_kernels.cuh"

namespace arp {

__global__ void correction_kernel(const cd* __restrict__ F, const cd* __restrict__ G, cd* __restrict__ V,
                                  cd* __restrict__ VT, int H, int K1v, BasisTabs tb) {
  corr_body(F, G, V, VT, blockIdx.x, H, K1v, tb);
}

__global__ void finish_kernel(const cd* __restrict__ Ge, const cd* __restrict__ V, cd* __restrict__ U,
                              cd* __restrict__ Gc, int H, int K1, int K1g, BasisTabs tb) {
  finish_body(Ge, V, U, Gc, blockIdx.x, H, K1, K1g, tb);
}

__global__ void finish_change_kernel(const cd* __restrict__ Ge, const cd* __restrict__ V, cd* __restrict__ U,
                                     cd* __restrict__ Gc, const cd* __restrict__ Uold, double* __restrict__ rel, int H,
                                     int K1, int K1g, BasisTabs tb) {
  const int n = blockIdx.x;
  finish_body(Ge, V, U, Gc, n, H, K1, K1g, tb);
  if (!Uold) return;
  __syncthreads();  // the block's stores of U_{n+1}, visible to its threads
  const size_t o1 = (size_t)(n + 1) * 3 * H;
  const double r = slice_change_body(U + o1, Uold + o1, H);
  if (threadIdx.x == 0) rel[n + 1] = r;
}

__global__ void slice_change_kernel(const cd* __restrict__ U, const cd* __restrict__ Uold, double* __restrict__ rel,
                                    int H) {
  const int n = blockIdx.x + 1;
  const double r = slice_change_body(U + (size_t)n * 3 * H, Uold + (size_t)n * 3 * H, H);
  if (threadIdx.x == 0) rel[n] = r;
}

__global__ void max_kernel(const double* __restrict__ rel, int S, double* __restrict__ out) {
  const double m = max_change_body(rel, S);
  if (threadIdx.x == 0) out[0] = m;
}

namespace {

BasisTabs basis_tabs(const arp_ctx* c) { return BasisTabs{c->inv_sig64, c->sk_sig64, c->dhalf}; }

// G(U_n) for the single state at U + n, written to g_out; u_next = g (+ v), with
// one launch per step of the link (used when the persistent chain cannot be
// co-resident).
arp_status chain_link(arp_ctx* c, const cd* u, cd* g_out, cd* u_next, const cd* v, cudaStream_t s) {
  arp_status r;
  if ((r = launch_to_eigen(c, u, c->W, 1, true, s)) != ARP_OK) return r;
  if ((r = launch_nbar_partial(c, c->W, c->partial, 1, s)) != ARP_OK) return r;
  if ((r = launch_nbar_reduce(c, kReduceMid, c->partial, c->W, c->W2, nullptr, nullptr, nullptr, 1, s)) != ARP_OK)
    return r;
  if ((r = launch_nbar_partial(c, c->W2, c->partial, 1, s)) != ARP_OK) return r;
  return launch_nbar_reduce(c, kReduceFinal, c->partial, c->W, nullptr, g_out, v, u_next, 1, s);
}

}  // namespace

// Reads the chain's status word; ARP_ETIMEOUT if a bounded wait (a grid
// barrier, or a cluster CTA's wait for data) gave up.
arp_status chain_status(arp_ctx* c, unsigned status) {
  if (status == 0u) return ARP_OK;
  return fail(c, ARP_ETIMEOUT, "chain: a bounded wait timed out (a block's arrival or data never came)");
}

// The whole serial chain n = 0..S-1: one thread-block cluster (then the
// parallel finish: U and the G cache from the eigen-basis g_n), else the
// persistent cooperative kernel, else one link at a time; in FP64 the
// cooperative kernel is tried first (ARP_OPT_CHAIN restricts the choice; the
// timeout test hook takes the cooperative kernel for value 1, whose grid
// barriers are the bounded waits it exercises, and the cluster for value 2).  V, if not
// null, is c->V, whose eigen form c->VT the correction kernel wrote with it.
arp_status run_chain(arp_ctx* c, const cd* V, cudaStream_t s) {
  const size_t st = (size_t)3 * c->H;
  // barrier counter and status word start at zero whichever kernel runs
  arp_status r = check_cuda(c, cudaMemsetAsync(c->sync, 0, 4 * sizeof(unsigned), s), "chain: status reset");
  if (r != ARP_OK) return r;
  if (c->coarse_grid) {
    // the asymptotic chain on the N_c grid (its sub-context's tables), from U_0
    // restricted to the coarse modes; the finish prolongs g_n back onto N
    if (c->coarse_scheme != 0 || (c->chain_mode != 0 && c->chain_mode != 3) || c->skip_arrival)
      return fail(c, ARP_EINVAL, "coarse grid: needs the asymptotic coarse scheme and the cluster chain");
    arp_ctx* q = c->coarse;
    if ((r = check_cuda(c, cudaMemcpy2DAsync(q->U, q->H * sizeof(cd), c->U, c->H * sizeof(cd), q->H * sizeof(cd), 3,
                                             cudaMemcpyDeviceToDevice, s), "coarse grid: restrict u0")) != ARP_OK)
      return r;
    if ((r = check_cuda(c, cudaMemsetAsync(q->sync, 0, 4 * sizeof(unsigned), s), "coarse grid: status reset")) !=
        ARP_OK)
      return r;
    r = launch_cluster_chain(q, q->U, q->Ge, V ? q->VT : nullptr, s);
    if (r != ARP_OK) return r == ARP_EINVAL ? fail(c, r, "coarse grid: no cluster chain fits") : fail(c, r, q->err);
    // the sub-context's chain status into this context's word, which the caller reads
    if ((r = check_cuda(c, cudaMemcpyAsync(c->sync + 1, q->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToDevice, s),
                        "coarse grid: status")) != ARP_OK)
      return r;
    finish_kernel<<<c->slices, 256, 0, s>>>(q->Ge, V, c->U, c->Gc, c->H, c->K1, q->K1, basis_tabs(c));
    return check_cuda(c, cudaGetLastError(), "chain: finish");
  }
  if (c->coarse_scheme == 1) return launch_strang_chain(c, c->U, c->Gc, V, s);
  r = ARP_EINVAL;
  // In FP64 with more than 16 nodes the chain's transforms are bound by GB300's
  // FP64 throughput, so the cooperative grid (up to one node per SM) comes
  // first; otherwise the cluster.
  if (fp64_grid_first(c) && !c->skip_arrival) r = launch_chain(c, c->U, c->Gc, V, s);
  if (r != ARP_EINVAL) return r;
  if ((c->chain_mode == 0 || c->chain_mode == 3) && c->skip_arrival != 1) {
    r = launch_cluster_chain(c, c->U, c->Ge, V ? c->VT : nullptr, s);
    if (r == ARP_OK) {
      finish_kernel<<<c->slices, 256, 0, s>>>(c->Ge, V, c->U, c->Gc, c->H, c->K1, c->K1, basis_tabs(c));
      r = check_cuda(c, cudaGetLastError(), "chain: finish");
    }
  }
  if (r != ARP_EINVAL) return r;
  if (c->chain_mode == 3) return fail(c, ARP_EINVAL, "chain: no cluster chain fits (ARP_OPT_CHAIN 3)");
  if (c->chain_mode <= 1) r = launch_chain(c, c->U, c->Gc, V, s);
  if (r != ARP_EINVAL) return r;
  for (int n = 0; n < c->slices; ++n)
    if ((r = chain_link(c, c->U + n * st, c->Gc + n * st, c->U + (n + 1) * st, V ? V + n * st : nullptr, s)) !=
        ARP_OK)
      return r;
  return ARP_OK;
}

arp_status parareal_iterate(arp_ctx* c, cudaStream_t s, int* k_done, double* change) {
  const size_t st = (size_t)3 * c->H;  // complex entries per state
  const int S = c->slices;
  arp_status r;
  if ((r = ensure_coarse(c, s)) != ARP_OK) return r;
  if (c->level < 0) {
    // predictor: U_{n+1} = G(U_n), G cached
    if ((r = run_chain(c, nullptr, s)) != ARP_OK) return r;
    unsigned status = 0;
    if ((r = check_cuda(c, cudaMemcpyAsync(&status, c->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                        "chain: status read")) != ARP_OK)
      return r;
    if ((r = check_cuda(c, cudaStreamSynchronize(s), "chain: synchronise")) != ARP_OK) return r;
    if ((r = chain_status(c, status)) != ARP_OK) return r;
    c->level = 0;
    if (k_done) *k_done = 0;
    if (change) *change = INFINITY;
    return ARP_OK;
  }
  std::swap(c->U, c->Uold);
  if ((r = launch_fine(c, c->Uold, c->Fb, S, s)) != ARP_OK) return r;
  {
    cd* vt = c->coarse_grid ? c->coarse->VT : c->VT;
    const int k1v = c->coarse_grid ? c->coarse->K1 : c->K1;
    correction_kernel<<<S, 256, 0, s>>>(c->Fb, c->Gc, c->V, vt, c->H, k1v, basis_tabs(c));
  }
  if ((r = check_cuda(c, cudaGetLastError(), "correction: launch")) != ARP_OK) return r;
  if ((r = check_cuda(c, cudaMemcpyAsync(c->U, c->Uold, st * sizeof(cd), cudaMemcpyDeviceToDevice, s),
                      "copy u0")) != ARP_OK)
    return r;
  if ((r = run_chain(c, c->V, s)) != ARP_OK) {
    std::swap(c->U, c->Uold);
    return r;
  }
  slice_change_kernel<<<S, 256, 0, s>>>(c->U, c->Uold, c->rel, c->H);
  max_kernel<<<1, 256, 0, s>>>(c->rel, S, c->scalar);
  if ((r = check_cuda(c, cudaGetLastError(), "norm: launch")) != ARP_OK) return r;
  double h = 0.0;
  unsigned status = 0;
  if ((r = check_cuda(c, cudaMemcpyAsync(&h, c->scalar, sizeof(double), cudaMemcpyDeviceToHost, s), "norm: read")) !=
      ARP_OK)
    return r;
  if ((r = check_cuda(c, cudaMemcpyAsync(&status, c->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                      "chain: status read")) != ARP_OK)
    return r;
  if ((r = check_cuda(c, cudaStreamSynchronize(s), "norm: synchronise")) != ARP_OK) return r;
  if ((r = chain_status(c, status)) != ARP_OK) {
    std::swap(c->U, c->Uold);
    return r;
  }
  c->level += 1;
  if (k_done) *k_done = c->level;
  if (change) *change = h;
  if (!std::isfinite(h)) return fail(c, ARP_ENONFINITE, "parareal: relative change is not finite");
  return ARP_OK;
}

}  // namespace arp

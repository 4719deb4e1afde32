// chain64.cu -- FP64 instantiations of the coarse-chain kernels (persistent
// cooperative grid, thread-block cluster) and their precision dispatch.
#include "chain_impl.cuh"
#include "cluster_chain.cuh"

namespace arp {

arp_status launch_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s);
arp_status launch_cluster_chain_f32(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                    const ChainRange* rg);

arp_status launch_cluster_chain(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                const ChainRange* rg) {
  if (c->precision != ARP_FP64) return launch_cluster_chain_f32(c, U0, Ge, VT, s, rg);
  return launch_cluster_chain_prec<double>(c, U0, Ge, VT, s, rg);
}

arp_status launch_chain(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  if (c->precision != ARP_FP64) return launch_chain_f32(c, U, Gc, V, s);
  return launch_chain_prec<double>(c, U, Gc, V, s);
}

}  // namespace arp

extern "C" arp_status arp_chain_exchange_bytes(int N, int cluster, int rank, int precision, unsigned* red_bytes,
                                               unsigned* ws_bytes) {
  using namespace arp;
  if (N < 8 || N > 2048 || (N & (N - 1)) != 0 || cluster < 1 || cluster > 16 || rank < 0 || rank >= cluster ||
      (precision != ARP_FP64 && precision != ARP_FP32) || !red_bytes || !ws_bytes)
    return ARP_EINVAL;
  int logn = 0;
  while ((1 << logn) < N) ++logn;
  const int K1 = (N - 1) / 3 + 1;
  // the ownership split of the launch plan (the node count does not enter it)
  const int own = precision == ARP_FP64 ? cluster_plan<double>(logn, 2, K1, cluster).own
                                        : cluster_plan<float>(logn, 2, K1, cluster).own;
  const ChainExchangeBytes xb =
      chain_exchange_bytes(K1, cluster, rank, own, precision == ARP_FP64 ? (int)sizeof(cd) : (int)sizeof(cf));
  *red_bytes = xb.red;
  *ws_bytes = xb.ws;
  return ARP_OK;
}

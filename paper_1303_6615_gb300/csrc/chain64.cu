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

// chain32.cu -- FP32 instantiations of the coarse-chain kernels.
#include "chain_impl.cuh"
#include "cluster_chain.cuh"

namespace arp {

arp_status launch_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  return launch_chain_prec<float>(c, U, Gc, V, s);
}

arp_status launch_cluster_chain_f32(arp_ctx* c, const cd* U0, cd* Ge, const cd* VT, cudaStream_t s,
                                    const ChainRange* rg) {
  return launch_cluster_chain_prec<float>(c, U0, Ge, VT, s, rg);
}

}  // namespace arp

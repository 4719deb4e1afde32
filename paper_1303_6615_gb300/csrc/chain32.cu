// chain32.cu -- FP32 instantiation of the persistent coarse-chain kernel.
#include "chain_impl.cuh"

namespace arp {

arp_status launch_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  return launch_chain_prec<float>(c, U, Gc, V, s);
}

}  // namespace arp

// chain64.cu -- FP64 instantiation of the persistent coarse-chain kernel and
// the precision dispatch.
#include "chain_impl.cuh"

namespace arp {

arp_status launch_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s);

arp_status launch_chain(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  if (c->precision == ARP_FP32) return launch_chain_f32(c, U, Gc, V, s);
  return launch_chain_prec<double>(c, U, Gc, V, s);
}

}  // namespace arp

// strang64.cu -- FP64 instantiations of the Strang kernels and the precision dispatch.
#include "strang_dispatch.cuh"

namespace arp {

arp_status launch_strang_sweep_f32(arp_ctx* c, const cd* in, cd* out, int batch, bool coarse, cudaStream_t s);
arp_status launch_strang_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s);

arp_status launch_strang_sweep(arp_ctx* c, const cd* in, cd* out, int batch, bool coarse, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  if (c->precision != ARP_FP64) return launch_strang_sweep_f32(c, in, out, batch, coarse, s);
  return launch_strang_sweep_prec<double>(c, in, out, batch, coarse, s);
}

arp_status launch_strang_chain(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  if (c->precision != ARP_FP64) return launch_strang_chain_f32(c, U, Gc, V, s);
  return launch_strang_chain_prec<double>(c, U, Gc, V, s);
}

}  // namespace arp

// strang32.cu -- FP32 instantiations of the Strang kernels.
#include "strang_dispatch.cuh"

namespace arp {

arp_status launch_strang_sweep_f32(arp_ctx* c, const cd* in, cd* out, int batch, bool coarse, cudaStream_t s) {
  return launch_strang_sweep_prec<float>(c, in, out, batch, coarse, s);
}

arp_status launch_strang_chain_f32(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  return launch_strang_chain_prec<float>(c, U, Gc, V, s);
}

}  // namespace arp

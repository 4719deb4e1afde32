// fine32.cu -- FP32 instantiations of the fine sweep and of the time-average kernel.
#include "coarse_impl.cuh"

namespace arp {

arp_status launch_fine_f32(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  return launch_fine_prec<float>(c, in, out, batch, s);
}

arp_status launch_nbar_f32(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  return launch_nbar_prec<float>(c, W, partial, batch, s);
}

}  // namespace arp

// ifrk32.cu -- FP32 instantiations of the integrating-factor RK4 fine sweep.
#include "fine_impl.cuh"

namespace arp {

arp_status launch_fine_ifrk4_f32(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  return launch_fine_prec<float, kSchemeIfrk4>(c, in, out, batch, s);
}

}  // namespace arp

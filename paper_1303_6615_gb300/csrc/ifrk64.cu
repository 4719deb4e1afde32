// ifrk64.cu -- FP64 instantiations of the integrating-factor RK4 fine sweep.
#include "fine_impl.cuh"

namespace arp {

arp_status launch_fine_ifrk4_f64(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  return launch_fine_prec<double, kSchemeIfrk4>(c, in, out, batch, s);
}

}  // namespace arp

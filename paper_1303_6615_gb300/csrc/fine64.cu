// fine64.cu -- FP64 instantiations of the fine sweep and of the time-average
// kernel, and the precision dispatch of both.
#include "coarse_impl.cuh"

namespace arp {

arp_status launch_fine_f32(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
arp_status launch_fine_ifrk4_f64(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
arp_status launch_fine_ifrk4_f32(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s);
arp_status launch_nbar_f32(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s);

arp_status launch_fine(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  if (c->fine_scheme == 1) return launch_strang_sweep(c, in, out, batch, false, s);
  if (c->fine_scheme == 2)
    return c->precision != ARP_FP64 ? launch_fine_ifrk4_f32(c, in, out, batch, s)
                                    : launch_fine_ifrk4_f64(c, in, out, batch, s);
  if (dft_mode(c)) return dft_fine(c, in, out, batch, s);
  if (c->precision == ARP_FP32) return launch_fine_f32(c, in, out, batch, s);
  return launch_fine_prec<double>(c, in, out, batch, s);
}

arp_status launch_nbar_partial(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  if (batch == 0) return ARP_OK;
  if (dft_mode(c)) return dft_nbar(c, W, partial, batch, s);
  if (c->precision == ARP_FP32) return launch_nbar_f32(c, W, partial, batch, s);
  return launch_nbar_prec<double>(c, W, partial, batch, s);
}

}  // namespace arp

// fine32.cu -- FP32 instantiations of the fine sweep and of the time-average kernel.
#include "coarse_impl.cuh"

namespace arp {

arp_status launch_fine_f32(arp_ctx* c, const cd* in, cd* out, int batch, cudaStream_t s) {
  return launch_fine_prec<float>(c, in, out, batch, s);
}

arp_status launch_nbar_f32(arp_ctx* c, const cd* W, cd* partial, int batch, cudaStream_t s) {
  return launch_nbar_prec<float>(c, W, partial, batch, s);
}

// The FP32 ETDRK4 fine sweep's schedule in effect for context c (1, 2 or 3).
int fine_schedule_in_effect(const arp_ctx* c) {
  switch (c->logN) {
    case 3: return fine_schedule_f32<3>(c);
    case 4: return fine_schedule_f32<4>(c);
    case 5: return fine_schedule_f32<5>(c);
    case 6: return fine_schedule_f32<6>(c);
    case 7: return fine_schedule_f32<7>(c);
    case 8: return fine_schedule_f32<8>(c);
    case 9: return fine_schedule_f32<9>(c);
    case 10: return fine_schedule_f32<10>(c);
    default: return fine_schedule_f32<11>(c);
  }
}

}  // namespace arp

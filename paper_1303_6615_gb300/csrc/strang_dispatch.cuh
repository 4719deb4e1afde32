// strang_dispatch.cuh -- table views and grid-size dispatch of the Strang
// kernels for one precision (instantiated in strang64.cu and strang32.cu).
#pragma once

#include "strang_impl.cuh"

namespace arp {

// Fine steps of size h: e^{lambda h} between steps (the ETDRK4 table E and, on
// the FP32 path, its low part), e^{lambda h/2} (the ETDRK4 table E2, FP64) at
// the ends.  Coarse step of size dT: e^{lambda dT/2} from its own table.
template <typename T>
StrangTabs<T> strang_tabs(const arp_ctx* c, bool coarse) {
  const int n = 3 * c->K1;
  StrangTabs<T> tb;
  if constexpr (std::is_same<T, float>::value) {
    tb.Ef = c->etd32;
    tb.Ef_lo = c->E_lo32;
    tb.tw = c->tw32;
    tb.is = c->inv_sig32;
    tb.ss = c->sk_sig32;
  } else {
    tb.Ef = c->etd64;
    tb.Ef_lo = nullptr;
    tb.tw = c->tw64;
    tb.is = c->inv_sig64;
    tb.ss = c->sk_sig64;
  }
  tb.Eh64 = coarse ? c->strang_h64 : c->etd64 + n;
  tb.is64 = c->inv_sig64;
  tb.ss64 = c->sk_sig64;
  tb.h = coarse ? c->dT : c->h;
  return tb;
}

template <typename T>
arp_status launch_strang_sweep_prec(arp_ctx* c, const cd* in, cd* out, int batch, bool coarse, cudaStream_t s) {
  const StrangTabs<T> tb = strang_tabs<T>(c, coarse);
  const int steps = coarse ? 1 : c->steps;
  switch (c->logN) {
    case 3: return launch_strang_sweep_n<T, 3>(c, in, out, batch, steps, tb, s);
    case 4: return launch_strang_sweep_n<T, 4>(c, in, out, batch, steps, tb, s);
    case 5: return launch_strang_sweep_n<T, 5>(c, in, out, batch, steps, tb, s);
    case 6: return launch_strang_sweep_n<T, 6>(c, in, out, batch, steps, tb, s);
    case 7: return launch_strang_sweep_n<T, 7>(c, in, out, batch, steps, tb, s);
    case 8: return launch_strang_sweep_n<T, 8>(c, in, out, batch, steps, tb, s);
    case 9: return launch_strang_sweep_n<T, 9>(c, in, out, batch, steps, tb, s);
    case 10: return launch_strang_sweep_n<T, 10>(c, in, out, batch, steps, tb, s);
    case 11: return launch_strang_sweep_n<T, 11>(c, in, out, batch, steps, tb, s);
    default: return fail(c, ARP_EINVAL, "strang: unsupported grid size");
  }
}

template <typename T>
arp_status launch_strang_chain_prec(arp_ctx* c, cd* U, cd* Gc, const cd* V, cudaStream_t s) {
  const StrangTabs<T> tb = strang_tabs<T>(c, true);
  switch (c->logN) {
    case 3: return launch_strang_chain_n<T, 3>(c, U, Gc, V, tb, s);
    case 4: return launch_strang_chain_n<T, 4>(c, U, Gc, V, tb, s);
    case 5: return launch_strang_chain_n<T, 5>(c, U, Gc, V, tb, s);
    case 6: return launch_strang_chain_n<T, 6>(c, U, Gc, V, tb, s);
    case 7: return launch_strang_chain_n<T, 7>(c, U, Gc, V, tb, s);
    case 8: return launch_strang_chain_n<T, 8>(c, U, Gc, V, tb, s);
    case 9: return launch_strang_chain_n<T, 9>(c, U, Gc, V, tb, s);
    case 10: return launch_strang_chain_n<T, 10>(c, U, Gc, V, tb, s);
    case 11: return launch_strang_chain_n<T, 11>(c, U, Gc, V, tb, s);
    default: return fail(c, ARP_EINVAL, "strang chain: unsupported grid size");
  }
}

}  // namespace arp

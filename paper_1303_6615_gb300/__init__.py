"""GB300-native asymptotic parareal for the 1D rotating shallow-water system.

The compute path is the CUDA library libarp.so (C ABI in include/arp.h),
built in-tree by `paper_1303_6615_gb300.build`; `paper_1303_6615_gb300.binding`
marshals torch device memory and streams into it.
"""
from .binding import (ARP_FP32, ARP_FP64, ARP_OPT_F, ARP_OPT_KMAX, ARP_OPT_PRECISION, ARP_OPT_T0,
                      ARP_OPT_TOL, ArpError, Solver, arp_coarse_avg, arp_coarse_step, arp_create,
                      arp_destroy, arp_fine_batch, arp_get_slices, arp_info, arp_last_error,
                      arp_parareal_iterate, arp_parareal_solve, arp_query_bytes, arp_set_initial,
                      arp_set_option, load_library)

__all__ = [
    "ARP_FP32", "ARP_FP64", "ARP_OPT_F", "ARP_OPT_KMAX", "ARP_OPT_PRECISION", "ARP_OPT_T0", "ARP_OPT_TOL",
    "ArpError", "Solver", "arp_coarse_avg", "arp_coarse_step", "arp_create", "arp_destroy",
    "arp_fine_batch", "arp_get_slices", "arp_info", "arp_last_error", "arp_parareal_iterate",
    "arp_parareal_solve", "arp_query_bytes", "arp_set_initial", "arp_set_option", "load_library",
]

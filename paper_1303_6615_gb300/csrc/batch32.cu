// batch32.cu -- FP32 instantiations of the fused multi-problem launches.
#include "batch_impl.cuh"

namespace arp {

arp_status launch_fine_batch_f32(arp_ctx* err, arp_ctx* tune, int logN, const void* jobs, const int* first, int njobs, int nblocks,
                                    cudaStream_t s) {
  switch (logN) {
    case 3: return launch_fine_batch_n<float, 3>(err, tune, jobs, first, njobs, nblocks, s);
    case 4: return launch_fine_batch_n<float, 4>(err, tune, jobs, first, njobs, nblocks, s);
    case 5: return launch_fine_batch_n<float, 5>(err, tune, jobs, first, njobs, nblocks, s);
    case 6: return launch_fine_batch_n<float, 6>(err, tune, jobs, first, njobs, nblocks, s);
    case 7: return launch_fine_batch_n<float, 7>(err, tune, jobs, first, njobs, nblocks, s);
    case 8: return launch_fine_batch_n<float, 8>(err, tune, jobs, first, njobs, nblocks, s);
    case 9: return launch_fine_batch_n<float, 9>(err, tune, jobs, first, njobs, nblocks, s);
    case 10: return launch_fine_batch_n<float, 10>(err, tune, jobs, first, njobs, nblocks, s);
    case 11: return launch_fine_batch_n<float, 11>(err, tune, jobs, first, njobs, nblocks, s);
    default: return fail(err, ARP_EINVAL, "batch fine: unsupported grid size");
  }
}

arp_status plan_chain_batch_f32(int logN, const int* M, const int* K1, int count, int* C, ClusterPlan* plans,
                                   size_t* smem) {
  switch (logN) {
    case 3: return plan_chain_batch_n<float, 3>(M, K1, count, C, plans, smem);
    case 4: return plan_chain_batch_n<float, 4>(M, K1, count, C, plans, smem);
    case 5: return plan_chain_batch_n<float, 5>(M, K1, count, C, plans, smem);
    case 6: return plan_chain_batch_n<float, 6>(M, K1, count, C, plans, smem);
    case 7: return plan_chain_batch_n<float, 7>(M, K1, count, C, plans, smem);
    case 8: return plan_chain_batch_n<float, 8>(M, K1, count, C, plans, smem);
    case 9: return plan_chain_batch_n<float, 9>(M, K1, count, C, plans, smem);
    case 10: return plan_chain_batch_n<float, 10>(M, K1, count, C, plans, smem);
    case 11: return plan_chain_batch_n<float, 11>(M, K1, count, C, plans, smem);
    default: return ARP_EINVAL;
  }
}

arp_status launch_chain_batch_f32(arp_ctx* err, int logN, const void* jobs, int count, int C, size_t smem,
                                     cudaStream_t s) {
  switch (logN) {
    case 3: return launch_chain_batch_n<float, 3>(err, jobs, count, C, smem, s);
    case 4: return launch_chain_batch_n<float, 4>(err, jobs, count, C, smem, s);
    case 5: return launch_chain_batch_n<float, 5>(err, jobs, count, C, smem, s);
    case 6: return launch_chain_batch_n<float, 6>(err, jobs, count, C, smem, s);
    case 7: return launch_chain_batch_n<float, 7>(err, jobs, count, C, smem, s);
    case 8: return launch_chain_batch_n<float, 8>(err, jobs, count, C, smem, s);
    case 9: return launch_chain_batch_n<float, 9>(err, jobs, count, C, smem, s);
    case 10: return launch_chain_batch_n<float, 10>(err, jobs, count, C, smem, s);
    case 11: return launch_chain_batch_n<float, 11>(err, jobs, count, C, smem, s);
    default: return fail(err, ARP_EINVAL, "batch chain: unsupported grid size");
  }
}

}  // namespace arp

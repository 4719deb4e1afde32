// batch_impl.cuh -- fused launches over many independent problems (contexts of
// the same grid size and precision): the fine sweep of every (problem, slice)
// pair in one launch, and the serial coarse chains of all problems in one
// launch of one thread-block cluster per problem.  The blocks run the same
// device bodies as the single-problem kernels, so a problem's results do not
// depend on which other problems share the launch.
#pragma once

#include <type_traits>

#include "cluster_chain.cuh"

namespace arp {

template <typename T>
struct FineJob {
  const cd* in;   // [slices][3][H]
  cd* out;        // [slices][3][H]
  int steps;
  FineTabs<T> tb;
};

template <typename T>
struct ChainJob {
  ClusterChainArgs a;
  NbarTabs<T> tb;
};

// Index of the job owning block b: the last i with first[i] <= b (first ascending).
__device__ __forceinline__ int find_job(const int* __restrict__ first, int njobs, int b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) fine_batch_kernel(const FineJob<T>* __restrict__ jobs,
                                                           const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const FineJob<T> j = jobs[i];
  if constexpr (std::is_same<T, float>::value)
    fine_f32_body<LOGN, BLOCK>(j.in, j.out, j.steps, j.tb, blockIdx.x - first[i]);
  else
    fine_body<T, LOGN, BLOCK>(j.in, j.out, j.steps, j.tb, blockIdx.x - first[i]);
}

// The lane-pair FP32 schedule over many problems (launch bounds as its single-problem kernel).
template <int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK, fine_pairs_min_blocks<LOGN>())
    fine_batch_kernel_pairs(const FineJob<float>* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const FineJob<float> j = jobs[i];
  fine_f32_body<LOGN, BLOCK, kSchemeEtdrk4, kPlanPairs>(j.in, j.out, j.steps, j.tb, blockIdx.x - first[i]);
}

// The radix-16 FP32 schedule over many problems.
template <int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK, fine_pairs_min_blocks<LOGN>())
    fine_batch_kernel_r16(const FineJob<float>* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int i = find_job(first, njobs, blockIdx.x);
  const FineJob<float> j = jobs[i];
  fine_f32_body<LOGN, BLOCK, kSchemeEtdrk4, kPlanRadix16>(j.in, j.out, j.steps, j.tb, blockIdx.x - first[i]);
}

template <typename T, int LOGN, int BLOCK>
__global__ void __launch_bounds__(BLOCK) chain_batch_kernel(const ChainJob<T>* __restrict__ jobs) {
  const int i = blockIdx.x / cooperative_groups::this_cluster().num_blocks();
  const ChainJob<T> j = jobs[i];
  chain_cluster_body<T, LOGN, BLOCK>(j.a, j.tb);
}

template <typename T, int LOGN, int BLOCK, int PLAN = kPlanRadix8>
arp_status launch_fine_batch_block(arp_ctx* err, const void* jobs, const int* first, int njobs, int nblocks,
                                   cudaStream_t s) {
  constexpr bool kF32 = std::is_same<T, float>::value;
  const size_t smem = kF32 ? F32Layout<LOGN, BLOCK, PLAN>::kBytes : FineLayout<T, LOGN>::kBytes;
  const void* kern;
  if constexpr (PLAN == kPlanRadix16) kern = (const void*)fine_batch_kernel_r16<LOGN, BLOCK>;
  else if constexpr (PLAN == kPlanPairs) kern = (const void*)fine_batch_kernel_pairs<LOGN, BLOCK>;
  else kern = (const void*)fine_batch_kernel<T, LOGN, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(err, e, "batch fine: shared-memory attribute");
  if constexpr (PLAN != kPlanRadix8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return check_cuda(err, e, "batch fine: shared-memory carveout");
  }
  void* args[] = {(void*)&jobs, (void*)&first, &njobs};
  return check_cuda(err, cudaLaunchKernel(kern, dim3(nblocks), dim3(BLOCK), args, smem, s), "batch fine: launch");
}

// `tune` is a member context of the group: its ARP_OPT_FINE_BLOCK (or the
// tuned per-size default) sets the FP32 schedule, as for one context.
template <typename T, int LOGN>
arp_status launch_fine_batch_n(arp_ctx* err, arp_ctx* tune, const void* jobs, const int* first, int njobs,
                               int nblocks, cudaStream_t s) {
  constexpr int B0 = FineBlock<LOGN>::value, B1 = FineBlockAlt<LOGN>::value;
  if constexpr (std::is_same<T, float>::value) {
    const int v = fine_schedule_f32<LOGN>(tune);
    if constexpr (r16_available(LOGN)) {
      if (v == 4)
        return launch_fine_batch_block<T, LOGN, FinePairBlock<LOGN>::value, kPlanRadix16>(err, jobs, first, njobs,
                                                                                         nblocks, s);
    }
    if constexpr (fine_pairs_available(LOGN)) {
      if (v == 3)
        return launch_fine_batch_block<T, LOGN, FinePairBlock<LOGN>::value, kPlanPairs>(err, jobs, first, njobs,
                                                                                       nblocks, s);
    }
    if constexpr (B0 != B1) {
      if (v == 2) return launch_fine_batch_block<T, LOGN, B1>(err, jobs, first, njobs, nblocks, s);
    }
  }
  return launch_fine_batch_block<T, LOGN, B0>(err, jobs, first, njobs, nblocks, s);
}

// Cluster chains of `count` problems of one grid size; `plans` gets each
// problem's plan for the chosen cluster size.  ARP_EINVAL (nothing launched)
// if some problem has no cluster plan.
template <typename T, int LOGN>
arp_status plan_chain_batch_n(const int* M, const int* K1, int count, int* C_out, ClusterPlan* plans,
                              size_t* smem_out) {
  constexpr int BLOCK = ClusterBlock<LOGN>::value;
  const void* kern = (const void*)chain_batch_kernel<T, LOGN, BLOCK>;
  for (int C : {16, 8}) {
    size_t smem = 0;
    bool ok = true;
    for (int i = 0; i < count && ok; ++i) {
      plans[i] = cluster_plan<T>(LOGN, M[i], K1[i], C);
      ok = plans[i].smem <= kMaxSmem;
      smem = plans[i].smem > smem ? plans[i].smem : smem;
    }
    if (!ok) continue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (!cluster_config(kern, C, BLOCK, smem, count, nullptr, &cfg, attr)) continue;
    *C_out = C;
    *smem_out = smem;
    return ARP_OK;
  }
  return ARP_EINVAL;
}

template <typename T, int LOGN>
arp_status launch_chain_batch_n(arp_ctx* err, const void* jobs, int count, int C, size_t smem, cudaStream_t s) {
  constexpr int BLOCK = ClusterBlock<LOGN>::value;
  const void* kern = (const void*)chain_batch_kernel<T, LOGN, BLOCK>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if (!cluster_config(kern, C, BLOCK, smem, count, s, &cfg, attr))
    return fail(err, ARP_EINVAL, "batch chain: cluster configuration not available");
  void* args[] = {(void*)&jobs};
  return check_cuda(err, cudaLaunchKernelExC(&cfg, kern, args), "batch chain: launch");
}

}  // namespace arp

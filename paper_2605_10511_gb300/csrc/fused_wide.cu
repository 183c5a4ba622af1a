// The fused kernel builds for CTAs of 512 threads (2 per SM) and 1,024
// threads (1 per SM): device-resident pages, no general string matcher.
// Their register budget is the 4 x 256-thread build's (64 per thread); a
// larger CTA shares one copy of the shared-memory join tables and meets at
// query switches with more warps.
#include "fused_kernel.cuh"

namespace dpf {

cudaError_t fused_wide_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  return L.threads > 512 ? launch_as<false, 1, false, false, 1024>(L, smem, tb, s)
                         : launch_as<false, 2, false, false, 512>(L, smem, tb, s);
}

int fused_wide_occupancy(int threads, size_t smem) {
  return threads > 512 ? occupancy_of<false, 1, false, false, 1024>(threads, smem)
                       : occupancy_of<false, 2, false, false, 512>(threads, smem);
}

}  // namespace dpf

// The fused kernel builds with the staging ring (device-resident pages, no
// general string matcher), 3 and 4 CTAs per SM: launched when the tuning
// asks for staging and some query's first step is staged.
#include "fused_kernel.cuh"

namespace dpf {

cudaError_t fused_stage_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  return L.min_blocks == kFusedMinBlocksHi ? launch_as<false, kFusedMinBlocksHi, false, true>(L, smem, tb, s)
                                           : launch_as<false, kFusedMinBlocksLo, false, true>(L, smem, tb, s);
}

int fused_stage_occupancy(int threads, size_t smem, int min_blocks) {
  return min_blocks == kFusedMinBlocksHi ? occupancy_of<false, kFusedMinBlocksHi, false, true>(threads, smem)
                                         : occupancy_of<false, kFusedMinBlocksLo, false, true>(threads, smem);
}

}  // namespace dpf

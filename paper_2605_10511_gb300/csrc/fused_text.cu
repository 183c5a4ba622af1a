// The fused kernel builds for device-resident pages with the general string
// matcher (CONTAINS, FSST), 3 and 4 CTAs per SM.
#include "fused_kernel.cuh"

namespace dpf {

cudaError_t fused_text_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  return L.min_blocks == kFusedMinBlocksHi ? launch_as<false, kFusedMinBlocksHi, true>(L, smem, tb, s)
                                           : launch_as<false, kFusedMinBlocksLo, true>(L, smem, tb, s);
}

int fused_text_occupancy(int threads, size_t smem, int min_blocks) {
  return min_blocks == kFusedMinBlocksHi ? occupancy_of<false, kFusedMinBlocksHi, true>(threads, smem)
                                         : occupancy_of<false, kFusedMinBlocksLo, true>(threads, smem);
}

}  // namespace dpf

// The fused kernel builds for device-resident pages without the general string
// matcher (no CONTAINS or FSST step in the batch), 3 and 4 CTAs per SM.
#include "fused_kernel.cuh"

namespace dpf {

cudaError_t fused_lean_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  return L.min_blocks == kFusedMinBlocksHi ? launch_as<false, kFusedMinBlocksHi, false>(L, smem, tb, s)
                                           : launch_as<false, kFusedMinBlocksLo, false>(L, smem, tb, s);
}

int fused_lean_occupancy(int threads, size_t smem, int min_blocks) {
  return min_blocks == kFusedMinBlocksHi ? occupancy_of<false, kFusedMinBlocksHi, false>(threads, smem)
                                         : occupancy_of<false, kFusedMinBlocksLo, false>(threads, smem);
}

}  // namespace dpf

// The fused kernel builds for pages in pinned host memory read over the host
// link (the string matcher included), 3 and 4 CTAs per SM.
#include "fused_kernel.cuh"

namespace dpf {

cudaError_t fused_host_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  return L.min_blocks == kFusedMinBlocksHi ? launch_as<true, kFusedMinBlocksHi, true>(L, smem, tb, s)
                                           : launch_as<true, kFusedMinBlocksLo, true>(L, smem, tb, s);
}

int fused_host_occupancy(int threads, size_t smem, int min_blocks) {
  return min_blocks == kFusedMinBlocksHi ? occupancy_of<true, kFusedMinBlocksHi, true>(threads, smem)
                                         : occupancy_of<true, kFusedMinBlocksLo, true>(threads, smem);
}

}  // namespace dpf

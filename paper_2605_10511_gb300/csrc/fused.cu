// Launch and occupancy of the fused kernel (fused_kernel.cuh): picks one of
// its six builds for a batch and sizes its dynamic shared memory.
#include "tile.cuh"

namespace dpf {

cudaError_t fused_lean_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s);
cudaError_t fused_text_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s);
cudaError_t fused_host_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s);
cudaError_t fused_stage_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s);
cudaError_t fused_wide_launch(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s);
int fused_wide_occupancy(int threads, size_t smem);
int fused_text_occupancy(int threads, size_t smem, int min_blocks);
int fused_host_occupancy(int threads, size_t smem, int min_blocks);
int fused_stage_occupancy(int threads, size_t smem, int min_blocks);

size_t fused_dynamic_smem(uint32_t acc_slots, size_t smem_tables, int threads, uint32_t stage_bw) {
  return ((acc_slots * sizeof(unsigned long long) + 15) & ~size_t(15)) + ((smem_tables + 15) & ~size_t(15)) +
         size_t(threads / 32) * (kListCap * sizeof(uint32_t) + stage_warp_bytes(stage_bw));
}

// The occupancy of the string-capable build bounds the grid of both builds
// (same launch bounds and shared memory; the lean build needs no more
// registers); a staged launch (stage_bw > 0) runs the staging build.
int fused_blocks_per_sm(int threads, uint32_t acc_slots, size_t smem_tables, bool host_data, int min_blocks,
                        uint32_t stage_bw) {
  const size_t smem = fused_dynamic_smem(acc_slots, smem_tables, threads, stage_bw);
  if (threads > 256) return fused_wide_occupancy(threads, smem);
  if (host_data) return fused_host_occupancy(threads, smem, min_blocks);
  return stage_bw ? fused_stage_occupancy(threads, smem, min_blocks) : fused_text_occupancy(threads, smem, min_blocks);
}

// Host-resident batches and batches with a CONTAINS or FSST step run the
// string-capable build; device-resident batches without one run the lean
// build, or the staging build when the batch is staged.
cudaError_t launch_fused(const FusedLaunch& L, cudaStream_t s) {
  const size_t smem = fused_dynamic_smem(L.acc_slots, L.smem_tables, L.threads, L.stage_bw);
  const uint32_t tb = uint32_t((L.smem_tables + 15) & ~size_t(15));
  if (L.threads > 256) return fused_wide_launch(L, smem, tb, s);  // prepare admits lean batches only
  if (L.host_data) return fused_host_launch(L, smem, tb, s);
  if (L.text) return fused_text_launch(L, smem, tb, s);
  if (L.stage_bw) return fused_stage_launch(L, smem, tb, s);
  return fused_lean_launch(L, smem, tb, s);
}

}  // namespace dpf

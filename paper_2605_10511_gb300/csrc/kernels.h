// Host-callable launchers of the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dpf_internal.h"

namespace dpf {

// Shared-memory accumulator capacity of one CTA (int64 slots).
constexpr uint32_t kSmemAccSlots = 4096;
constexpr uint32_t kMbPerWarpTile = 4;
// The fused kernel is compiled twice, for 3 and for 4 resident 256-thread CTAs
// per SM (register budgets of 80 and 64 per thread): occupancy, more than
// issue, bounds it.  The 4-CTA build spills a little and wins when four CTAs'
// shared memory fits; the launch configuration (ctas_per_sm) picks one.
constexpr int kFusedMinBlocksLo = 3;
constexpr int kFusedMinBlocksHi = 4;
// Rows of one scheduling ticket (one warp's unit of work) unless tuned.
constexpr uint32_t kDefaultChunkRows = 4096;
// Shared memory of one warp's survivor list (1,024 entries).
constexpr uint32_t kListBytesPerWarp = 1024 * 4;
// Estimated selectivity of the first step from which step 1's mini blocks
// are prefetched into L2 during the dense tiles (DevQuery::pf_step).
constexpr double kPrefetchMinSel = 0.03;
// Staging of the first step's mini blocks unless tuned (DPF_STAGE_ON / _OFF).
constexpr int32_t kDefaultStaging = 2;
// Grouped aggregates are added with one int64 atomic per row unless tuned
// (DPF_GROUP_AGG_*): warp aggregation measured slower on GB300 both with
// 1,024 Zipf groups (1.8x) and with 15 groups, one holding 97 % of the rows
// (1.3x); the autotuner tries it per plan signature.
constexpr int32_t kDefaultGroupAgg = 2;
// Join-table representation by the key range of the kept rows (R8): a
// direct table of one word per key up to 2^22 keys (16 MB), a rank
// directory (2 bits per key plus the kept payloads) up to 2^28 keys, open
// addressing beyond.
constexpr uint64_t kDirectMaxRange = uint64_t(1) << 22;
constexpr uint64_t kRankMaxRange = uint64_t(1) << 28;
// Shared-memory bytes of the code-level matcher tables of a PREFIX / CONTAINS
// step with a pattern of plen bytes on an FSST column: for every matcher
// state 0..plen, the next state after one symbol code (256 entries) and
// after one literal byte (256 entries).
inline uint32_t fsst_match_bytes(uint32_t plen) { return (plen + 1) * 512u; }

// Fused persistent kernel over a batch of compiled queries (Sec. 3.2).
// qbegin[0..nq] = first ticket of each query (qbegin[nq] = total tickets).
struct FusedLaunch {
  const DevQuery* queries;
  const uint64_t* qbegin;
  int nq;
  uint64_t total_chunks;
  Sched* sched;
  int grid, threads;
  uint32_t acc_slots;   // int64 shared accumulators per CTA (max over the batch)
  size_t smem_tables;   // bytes of the CTA's join-table region
  bool host_data;       // some column lives in mapped pinned host memory
  int min_blocks;       // kFusedMinBlocksLo or kFusedMinBlocksHi: which build runs
  bool text;            // some query has a CONTAINS step or a string step on an FSST
                        // column (the build with the general string matcher runs)
  uint32_t stage_bw;    // bits a value of the warps' staging ring slots hold; 0 = no ring
};
cudaError_t launch_fused(const FusedLaunch& L, cudaStream_t s);
// Occupancy of the fused kernel for (threads, dynamic smem); also sets the
// kernel's dynamic shared-memory limit.
int fused_blocks_per_sm(int threads, uint32_t acc_slots, size_t smem_tables, bool host_data, int min_blocks,
                        uint32_t stage_bw = 0);
size_t fused_dynamic_smem(uint32_t acc_slots, size_t smem_tables, int threads, uint32_t stage_bw = 0);

// Hash build (Kernel #1 of Sec. 3.1).  `q` describes the dimension scan:
// cols/steps as for the fused kernel, build_key/build_pay name columns.
struct BuildLaunch {
  const DevQuery* q;          // device copy
  uint2* table;               // open addressing: capacity slots (mask + 1)
  uint32_t mask;
  uint32_t* direct;           // direct table: krange entries (or nullptr)
  int32_t kmin;
  uint32_t krange;
  uint4* rank_dir;            // rank table: (krange + 63) / 64 directory words (or nullptr)
  uint32_t* rank_pay;         //   payloads of the present keys, in key order
  uint32_t* rank_sums;        //   scratch: one count per 1,024 directory words
  uint2* rank_stage;          //   scratch: {key offset, payload} of each inserted row, in insertion order
  unsigned long long* stage_n;  //   its count
  uint32_t rank_cap;          //   payload words (= staged pairs) the table holds
  unsigned long long* count;  // device counter (count pass)
  int32_t* kminmax;           // device {min, max} of kept keys (count pass)
  unsigned long long* inserted;  // tables sized before the scan: rows the insert pass kept (or nullptr)
  Sched* sched;               // status word
  uint64_t nrows, page_rows;
  bool host_data;
};
// Device-side outcome of a table sized before its scan: the build kernels'
// status bits and the rows the insert pass kept.
struct BuildStat {
  Sched sched;
  unsigned long long inserted;
};
cudaError_t launch_build_count(const BuildLaunch& L, cudaStream_t s);
cudaError_t launch_build_insert(const BuildLaunch& L, cudaStream_t s);
cudaError_t launch_init_table(uint2* table, uint32_t slots, cudaStream_t s);
cudaError_t launch_init_direct(uint32_t* table, uint32_t n, cudaStream_t s);

// Unfused per-operator chain (baseline).  Buffers for every intermediate:
// decoded columns, predicate flags, two ping-pong (row id, group id) lists
// and the device-side list lengths.
struct UnfusedChain {
  DevQuery q;                 // host copy of the compiled plan
  const DevQuery* dq;         // device copy (read by the assembly kernel)
  int32_t* vals[kMaxCols];    // decoded int columns
  int32_t* lens[kMaxCols];    // decoded string lengths
  uint64_t* offs[kMaxCols];   // absolute string byte offsets in the column blob
  uint8_t* flags;
  uint32_t* rid[2];
  uint32_t* gid[2];
  unsigned long long* counts; // [2 + kMaxSteps] list lengths
  Sched* sched;
};
constexpr int kUnfusedCounts = 2 + kMaxSteps;
cudaError_t launch_unfused(const UnfusedChain& U, cudaStream_t s, uint32_t* launches);

}  // namespace dpf

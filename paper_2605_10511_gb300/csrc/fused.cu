// The fused persistent kernel (Sec. 3.2, Sec. 4.1 "fused kernel composition").
//
// One launch executes every query of a batch.  Each CTA repeatedly takes a
// ticket (one chunk of one query's fact table: the outer loop of Sec. 3.2
// without host intervention), splits the chunk into warp tiles of
// TB mini blocks and runs decode -> predicates -> probes -> aggregation on
// them with all row state in registers.  Per-CTA int64 accumulators live in
// shared memory while the CTA stays on one query; they are added to the
// query's global accumulators when the CTA moves to another query or exits.
// The CTA that flushes a query's last chunk turns its accumulators into
// records ordered by key tuple (the record format of Kernel #3, Sec. 3.1) and
// zeroes the scratch state, so the kernel can be replayed from a CUDA graph.
#include "../../include/dpf.h"
#include "tile.cuh"

namespace dpf {
namespace {

struct alignas(16) CtaState {
  DevQuery q;
  unsigned long long ticket;
  int qi;
  int last;
  unsigned int warp_sum[32];
};

// Block-wide exclusive scan of a 0/1 flag; returns the rank, *total the sum.
__device__ __forceinline__ uint32_t block_rank(bool flag, CtaState& cs, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned b = __ballot_sync(kFull, flag);
  if (lane == 0) cs.warp_sum[warp] = __popc(b);
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int w = 0; w < nw; ++w) {
    const uint32_t x = cs.warp_sum[w];
    if (w < warp) before += x;
    all += x;
  }
  __syncthreads();
  *total = all;
  return before + __popc(b & ((1u << lane) - 1u));
}

// Converts a query's global accumulators into records and clears them.
__device__ void assemble(const DevQuery& Q, CtaState& cs) {
  const uint32_t S1 = 1 + Q.naggs;
  dpf_record* out = reinterpret_cast<dpf_record*>(Q.out);
  if (Q.nkeys == 0) {
    if (threadIdx.x == 0) {
      dpf_record r;
      r.key[0] = r.key[1] = 0;
      r.count = (long long)__ldcg(Q.acc);
      for (int a = 0; a < 4; ++a) r.val[a] = a < int(Q.naggs) ? (long long)__ldcg(Q.acc + 1 + a) : 0;
      out[0] = r;
      *Q.out_n = 1;
    }
  } else {
    uint32_t base = 0;
    for (uint32_t g0 = 0; g0 < Q.domain; g0 += blockDim.x) {
      const uint32_t g = g0 + threadIdx.x;
      const unsigned long long cnt = g < Q.domain ? __ldcg(Q.acc + uint64_t(g) * S1) : 0ull;
      uint32_t total;
      const uint32_t rank = block_rank(cnt != 0, cs, &total);
      if (cnt != 0) {
        dpf_record r;
        for (int k = 0; k < 2; ++k) {
          if (k < int(Q.nkeys)) {
            const uint32_t code = (g / Q.key_div[k]) % Q.key_dom[k];
            r.key[k] = __ldg(Q.key_dict[k] + code);
          } else {
            r.key[k] = 0;
          }
        }
        r.count = (long long)cnt;
        for (int a = 0; a < 4; ++a)
          r.val[a] = a < int(Q.naggs) ? (long long)__ldcg(Q.acc + uint64_t(g) * S1 + 1 + a) : 0;
        out[base + rank] = r;
      }
      base += total;
    }
    if (threadIdx.x == 0) *Q.out_n = base;
  }
  __syncthreads();
  const uint64_t n = uint64_t(Q.domain) * S1;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) Q.acc[i] = 0ull;
  if (threadIdx.x == 0) *Q.done = 0u;
  __threadfence();
}

// Adds the CTA's accumulators for Q to global memory, counts the chunks it
// processed and, if they were the query's last, assembles the result.
__device__ void finish_query(const DevQuery& Q, unsigned long long* sacc, uint32_t mine,
                             CtaState& cs) {
  const uint32_t S1 = 1 + Q.naggs;
  if (Q.use_smem_acc) {
    const uint32_t n = Q.domain * S1;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long x = sacc[i];
      if (x) atomicAdd(Q.acc + i, x);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned old = atomicAdd(Q.done, mine);
    cs.last = (uint64_t(old) + mine == Q.nchunks);
  }
  __syncthreads();
  if (cs.last) {
    __threadfence();
    assemble(Q, cs);
  }
  __syncthreads();
}

// Aggregation of a tile's live rows (Kernel #3 hash aggregation; int64 as
// in Sec. 4.3).  domain == 1: per-lane registers; otherwise int64 atomics
// into the CTA's shared accumulators (or global ones for large domains).
template <bool kHost>
__device__ __forceinline__ void tile_aggregate(const DevQuery& Q, TileState& T, int lane,
                                               unsigned long long* acc, long long (&racc)[5],
                                               unsigned int* status) {
  const uint32_t S1 = 1 + Q.naggs;
  const bool single = Q.domain == 1;
  if (!single) {
    // a corrupt dictionary code could push a group id out of the domain
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (((T.alive >> (4 * t + k)) & 1u) && T.gid[t][k] >= Q.domain) {
          T.alive &= ~(1u << (4 * t + k));
          atomicOr(status, S_CORRUPT);
        }
  }
  if (single) {
    racc[0] += __popc(T.alive);
  } else {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((T.alive >> (4 * t + k)) & 1u) atomicAdd(acc + uint64_t(T.gid[t][k]) * S1, 1ull);
  }
  for (uint32_t a = 0; a < Q.naggs; ++a) {
    const uint32_t op = Q.agg_op[a];
    uint32_t va[TB][4], vb[TB][4], anym;
    MbHdr H[TB];
    if (op != DPF_AGG_COUNT) tile_decode<kHost>(Q, Q.agg_a[a], T, lane, va, anym, H, status);
    if (op == DPF_AGG_SUM_MUL || op == DPF_AGG_SUM_SUB)
      tile_decode<kHost>(Q, Q.agg_b[a], T, lane, vb, anym, H, status);
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((T.alive >> (4 * t + k)) & 1u)) continue;
        long long x;
        if (op == DPF_AGG_COUNT) x = 1;
        else if (op == DPF_AGG_SUM) x = (long long)int32_t(va[t][k]);
        else if (op == DPF_AGG_SUM_MUL)
          x = (long long)((unsigned long long)(long long)int32_t(va[t][k]) *
                          (unsigned long long)(long long)int32_t(vb[t][k]));
        else x = (long long)int32_t(va[t][k]) - (long long)int32_t(vb[t][k]);
        if (single) racc[1 + a] += x;
        else atomicAdd(acc + uint64_t(T.gid[t][k]) * S1 + 1 + a, (unsigned long long)x);
      }
  }
}

// One ticket: the rows [chunk*chunk_rows, +chunk_rows) of Q's fact table,
// cut at page boundaries into warp tiles that the CTA's warps share.
template <bool kHost>
__device__ void process_chunk(const DevQuery& Q, uint64_t chunk, unsigned long long* acc,
                              const uint8_t* stab, unsigned int* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t P = Q.page_rows;
  const uint64_t r0 = chunk * Q.chunk_rows;
  const uint64_t r1 = min(Q.nrows, r0 + Q.chunk_rows);
  long long racc[5] = {0, 0, 0, 0, 0};
  uint64_t tile_base = 0;
  for (uint64_t p = r0 / P; p <= (r1 - 1) / P; ++p) {
    const uint64_t pr0 = max(r0, p * P), pr1 = min(r1, (p + 1) * P);
    const uint32_t mb0 = uint32_t((pr0 - p * P) / kMB);
    const uint32_t mb1 = uint32_t((pr1 - p * P + kMB - 1) / kMB);
    const uint32_t ntiles = (mb1 - mb0 + TB - 1) / TB;
    uint32_t j = uint32_t((warp + nw - int(tile_base % nw)) % nw);
    for (; j < ntiles; j += nw) {
      const uint32_t i0 = mb0 + j * TB;
      TileState T;
      tile_begin<kHost>(Q, p, i0, tmin<uint32_t>(TB, mb1 - i0), lane, T);
      if (tile_steps<kHost>(Q, T, stab, lane, status))
        tile_aggregate<kHost>(Q, T, lane, acc, racc, status);
    }
    tile_base += ntiles;
  }
  if (Q.domain == 1) {
    const uint32_t S1 = 1 + Q.naggs;
    for (uint32_t s = 0; s < S1; ++s) {
      long long x = racc[s];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(kFull, x, d);
      if (lane == 0 && x != 0) atomicAdd(acc + s, (unsigned long long)x);
    }
  }
}

template <bool kHost>
__global__ void __launch_bounds__(512) fused_kernel(const DevQuery* __restrict__ queries,
                                                     const uint64_t* __restrict__ qbegin, int nq,
                                                     uint64_t total, Sched* sched) {
  extern __shared__ __align__(16) uint8_t dyn[];
  __shared__ CtaState cs;
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(dyn);
  uint8_t* stab = dyn + kSmemAccSlots * sizeof(unsigned long long);
  int cur = -1;
  uint32_t mine = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(&sched->next, 1ull);
      int qi = -1;
      if (t < total) {
        int lo = 0, hi = nq - 1;  // last query with qbegin <= t
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if (__ldg(qbegin + mid) <= t) lo = mid; else hi = mid - 1;
        }
        qi = lo;
      }
      cs.ticket = t;
      cs.qi = qi;
    }
    __syncthreads();
    const unsigned long long t = cs.ticket;
    const int qi = cs.qi;
    if (qi != cur) {
      if (cur >= 0) finish_query(cs.q, sacc, mine, cs);
      if (qi < 0) break;
      {  // bring the query's plan into shared memory
        const uint4* src = reinterpret_cast<const uint4*>(queries + qi);
        uint4* dst = reinterpret_cast<uint4*>(&cs.q);
        for (uint32_t i = threadIdx.x; i < sizeof(DevQuery) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
      }
      __syncthreads();
      const DevQuery& Q = cs.q;
      if (Q.use_smem_acc) {
        const uint32_t n = Q.domain * (1 + Q.naggs);
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sacc[i] = 0ull;
      }
      for (uint32_t ti = 0; ti < Q.ntables; ++ti) {
        const SmemTable& st = Q.tables[ti];
        uint2* dst = reinterpret_cast<uint2*>(stab + st.offset);
        for (uint32_t i = threadIdx.x; i < st.slots; i += blockDim.x) dst[i] = __ldg(st.src + i);
      }
      __syncthreads();
      cur = qi;
      mine = 0;
    }
    const DevQuery& Q = cs.q;
    process_chunk<kHost>(Q, t - Q.chunk_begin, Q.use_smem_acc ? sacc : Q.acc, stab, &sched->status);
    ++mine;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&sched->exited, 1u);
    if (old == gridDim.x - 1) {
      sched->next = 0ull;
      sched->exited = 0u;
      __threadfence();
    }
  }
}

}  // namespace

size_t fused_dynamic_smem(size_t smem_tables) {
  return kSmemAccSlots * sizeof(unsigned long long) + smem_tables;
}

int fused_blocks_per_sm(int threads, size_t smem_tables, bool host_data) {
  const size_t smem = fused_dynamic_smem(smem_tables);
  int n = 0;
  if (host_data) {
    cudaFuncSetAttribute(fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel<true>, threads, smem);
  } else {
    cudaFuncSetAttribute(fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel<false>, threads, smem);
  }
  return n;
}

cudaError_t launch_fused(const FusedLaunch& L, cudaStream_t s) {
  const size_t smem = fused_dynamic_smem(L.smem_tables);
  if (L.host_data) {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<true><<<L.grid, L.threads, smem, s>>>(L.queries, L.qbegin, L.nq, L.total_chunks, L.sched);
  } else {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<false><<<L.grid, L.threads, smem, s>>>(L.queries, L.qbegin, L.nq, L.total_chunks, L.sched);
  }
  return cudaGetLastError();
}

}  // namespace dpf

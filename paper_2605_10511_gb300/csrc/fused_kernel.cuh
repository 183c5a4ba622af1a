// The fused persistent kernel (Sec. 3.2, Sec. 4.1 "fused kernel composition"),
// as a header: each of fused_lean.cu, fused_text.cu and fused_host.cu
// compiles two of its six builds (device-resident pages without / with the
// general string matcher, host-resident pages; 3 and 4 resident CTAs per
// SM each), so the builds compile in parallel.
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
#pragma once

#include <climits>

#include "../../include/dpf.h"
#include "tile.cuh"

namespace dpf {
namespace {

struct alignas(16) CtaState {
  DevQuery q;
  int wq[32];          // query of the ticket each warp holds (INT_MAX: none left)
  unsigned int mine;   // tickets of the current query this CTA processed
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

// Warp-aggregated group-by update (hash aggregation of Kernel #3, Sec. 3.1),
// by the round's leading group: the lanes holding the group id of the
// round's first valid lane combine their values with warp reductions and
// that lane issues the group's single atomic; every other valid lane adds
// its own value.  A hot group (a Zipf head, or one key holding most rows)
// thus costs one atomic per round instead of one per row on the same
// address.  The sum is exact modulo 2^64: a value is split into 16-bit parts
// whose sums over 32 lanes stay below 2^21 (kWide: four unsigned parts of
// the 64-bit value; otherwise the value is an int32, whose low 16 bits and
// signed high 16 bits are summed).  Warp-uniform call.
template <bool kWide>
__device__ __forceinline__ void lead_group_add(unsigned long long* acc, uint32_t gid, uint32_t S1, uint32_t slot,
                                               unsigned long long x, bool valid, int lane) {
  const uint32_t vm = __ballot_sync(kFull, valid);
  if (vm == 0) return;
  const int lead = __ffs(vm) - 1;
  const uint32_t g0 = __shfl_sync(kFull, gid, lead);
  const bool mine = valid && gid == g0;
  const uint32_t m = __ballot_sync(kFull, mine);
  if (mine) {
    unsigned long long t;
    if (kWide) {
      const uint32_t lo = uint32_t(x), hi = uint32_t(x >> 32);
      t = (unsigned long long)__reduce_add_sync(m, lo & 0xffffu) +
          ((unsigned long long)__reduce_add_sync(m, lo >> 16) << 16) +
          ((unsigned long long)__reduce_add_sync(m, hi & 0xffffu) << 32) +
          ((unsigned long long)__reduce_add_sync(m, hi >> 16) << 48);
    } else {
      const int32_t v = int32_t(uint32_t(x));
      const uint32_t s_lo = __reduce_add_sync(m, uint32_t(v) & 0xffffu);
      const int32_t s_hi = int32_t(__reduce_add_sync(m, uint32_t(v >> 16)));  // |sum| < 2^20
      t = (unsigned long long)((long long)s_lo + (long long)s_hi * 65536ll);
    }
    if (lane == lead) atomicAdd(acc + uint64_t(g0) * S1 + slot, t);
  } else if (valid) {
    atomicAdd(acc + uint64_t(gid) * S1 + slot, x);
  }
}

// A grouped update: warp-aggregated by the leading group (Q.warp_agg) or one
// atomic per row.
template <bool kWide>
__device__ __forceinline__ void group_add(const DevQuery& Q, unsigned long long* acc, uint32_t gid, uint32_t S1,
                                          uint32_t slot, unsigned long long x, bool valid, int lane) {
  if (Q.warp_agg) lead_group_add<kWide>(acc, gid, S1, slot, x, valid, lane);
  else if (valid) atomicAdd(acc + uint64_t(gid) * S1 + slot, x);
}

// One aggregate over a warp's list, specialised on its operation (dpf_agg_op)
// and on how its operands are read: kPoint = FOR/DICT columns, one bit field
// per row; otherwise any codec through row_value (DELTA decodes densely).
template <bool kHost, int kOp, bool kPoint>
__device__ __forceinline__ void agg_pass(const DevQuery& Q, const PageState& P, uint32_t seg_mb,
                                         const uint32_t* list, uint32_t n, int lane, unsigned long long* acc,
                                         uint32_t slot, int ca, int cb, bool single, unsigned int* status) {
  constexpr int U = kPoint ? kListUnroll : 1;  // rounds whose loads are issued together
  const uint32_t S1 = 1 + Q.naggs;
  long long sum = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += 32 * U) {
    uint32_t r[U], gid[U];
    bool valid[U];
    int32_t va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      valid[u] = i0 + 32u * u + lane < n;
      const uint32_t e = valid[u] ? list[i0 + 32u * u + lane] : 0u;
      r[u] = e & ((1u << kRowBits) - 1u);
      gid[u] = e >> kRowBits;
      if (!single && gid[u] >= Q.domain) valid[u] = false;  // reported by list_aggregate
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      va[u] = vb[u] = 0;
      if (kOp != DPF_AGG_COUNT)
        va[u] = int32_t(kPoint ? point_value<kHost>(Q, ca, P, seg_mb, r[u], valid[u])
                               : row_value<kHost>(Q, ca, P, seg_mb, r[u], valid[u], lane, status));
      if (kOp == DPF_AGG_SUM_MUL || kOp == DPF_AGG_SUM_SUB)
        vb[u] = int32_t(kPoint ? point_value<kHost>(Q, cb, P, seg_mb, r[u], valid[u])
                               : row_value<kHost>(Q, cb, P, seg_mb, r[u], valid[u], lane, status));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long x = 1;
      if (kOp == DPF_AGG_SUM) x = va[u];
      else if (kOp == DPF_AGG_SUM_MUL)
        x = (long long)((unsigned long long)(long long)va[u] * (unsigned long long)(long long)vb[u]);
      else if (kOp == DPF_AGG_SUM_SUB)
        x = (long long)va[u] - (long long)vb[u];
      if (single) sum += valid[u] ? x : 0;
      else group_add<kOp == DPF_AGG_SUM_MUL || kOp == DPF_AGG_SUM_SUB>(Q, acc, gid[u], S1, slot,
                                                                      (unsigned long long)x, valid[u], lane);
    }
  }
  if (single) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_down_sync(kFull, sum, d);
    if (lane == 0 && sum != 0) atomicAdd(acc + slot, (unsigned long long)sum);
  }
}

// An aggregate with a FOR64 operand: one survivor per lane, int64 operands,
// arithmetic modulo 2^64.  Inlined: an out-of-line call made the caller
// spill around it, while inlined it leaves the 32-bit passes' register
// allocation as it was.
template <bool kHost, int kOp>
__device__ __forceinline__ void agg_pass_wide(const DevQuery& Q, const PageState& P, uint32_t seg_mb,
                                           const uint32_t* list, uint32_t n, int lane, unsigned long long* acc,
                                           uint32_t slot, int ca, int cb, bool single, unsigned int* status) {
  const uint32_t S1 = 1 + Q.naggs;
  unsigned long long sum = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += 32) {
    bool valid = i0 + lane < n;
    const uint32_t e = valid ? list[i0 + lane] : 0u;
    const uint32_t r = e & ((1u << kRowBits) - 1u), gid = e >> kRowBits;
    if (!single && gid >= Q.domain) valid = false;  // reported by list_aggregate
    const unsigned long long a = (unsigned long long)value64<kHost>(Q, ca, P, seg_mb, r, valid, lane, status);
    unsigned long long b = 0;
    if (kOp == DPF_AGG_SUM_MUL || kOp == DPF_AGG_SUM_SUB)
      b = (unsigned long long)value64<kHost>(Q, cb, P, seg_mb, r, valid, lane, status);
    const unsigned long long x = kOp == DPF_AGG_SUM ? a : (kOp == DPF_AGG_SUM_MUL ? a * b : a - b);
    if (single) sum += valid ? x : 0ull;
    else group_add<true>(Q, acc, gid, S1, slot, x, valid, lane);
  }
  if (single) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_down_sync(kFull, sum, d);
    if (lane == 0 && sum != 0) atomicAdd(acc + slot, sum);
  }
}

template <bool kHost, int kOp>
__device__ __forceinline__ void agg_dispatch(const DevQuery& Q, const PageState& P, uint32_t seg_mb,
                                             const uint32_t* list, uint32_t n, int lane, unsigned long long* acc,
                                             uint32_t slot, int ca, int cb, bool single, unsigned int* status) {
  if (Q.cols[ca].codec == C_FOR64 || (kOp != DPF_AGG_SUM && Q.cols[cb].codec == C_FOR64)) {
    agg_pass_wide<kHost, kOp>(Q, P, seg_mb, list, n, lane, acc, slot, ca, cb, single, status);
    return;
  }
  const bool point = Q.cols[ca].codec != C_DELTA && (kOp == DPF_AGG_SUM || Q.cols[cb].codec != C_DELTA);
  if (point) agg_pass<kHost, kOp, true>(Q, P, seg_mb, list, n, lane, acc, slot, ca, cb, single, status);
  else agg_pass<kHost, kOp, false>(Q, P, seg_mb, list, n, lane, acc, slot, ca, cb, single, status);
}

// Aggregation over a warp's survivor list (Kernel #3 hash aggregation;
// int64 as in Sec. 4.3): slot 0 counts rows, slot 1 + a holds aggregate a.
// domain == 1: per-lane int64 sums reduced across the warp; otherwise
// int64 atomics (one per row, or warp-aggregated by the round's leading
// group: group_add) into the CTA's shared accumulators (or the query's
// global ones for large domains), indexed by the dense group id.
template <bool kHost>
__device__ __forceinline__ void list_aggregate(const DevQuery& Q, const PageState& P, uint32_t seg_mb,
                                               const uint32_t* list, uint32_t n, int lane,
                                               unsigned long long* acc, unsigned int* status) {
  const uint32_t S1 = 1 + Q.naggs;
  const bool single = Q.domain == 1;
  if (single) {
    if (lane == 0) atomicAdd(acc, (unsigned long long)n);
  } else {
    for (uint32_t i0 = 0; i0 < n; i0 += 32) {
      bool valid = i0 + lane < n;
      const uint32_t gid = valid ? list[i0 + lane] >> kRowBits : 0u;
      if (valid && gid >= Q.domain) {
        atomicOr(status, S_CORRUPT);  // a corrupt dictionary code
        valid = false;
      }
      group_add<false>(Q, acc, gid, S1, 0, 1ull, valid, lane);
    }
  }
  for (uint32_t a = 0; a < Q.naggs; ++a) {
    const int ca = Q.agg_a[a], cb = Q.agg_b[a];
    switch (Q.agg_op[a]) {
      case DPF_AGG_COUNT:
        if (single) {
          if (lane == 0) atomicAdd(acc + 1 + a, (unsigned long long)n);
        } else {
          agg_pass<kHost, DPF_AGG_COUNT, true>(Q, P, seg_mb, list, n, lane, acc, 1 + a, ca, cb, single, status);
        }
        break;
      case DPF_AGG_SUM:
        agg_dispatch<kHost, DPF_AGG_SUM>(Q, P, seg_mb, list, n, lane, acc, 1 + a, ca, cb, single, status);
        break;
      case DPF_AGG_SUM_MUL:
        agg_dispatch<kHost, DPF_AGG_SUM_MUL>(Q, P, seg_mb, list, n, lane, acc, 1 + a, ca, cb, single, status);
        break;
      default:
        agg_dispatch<kHost, DPF_AGG_SUM_SUB>(Q, P, seg_mb, list, n, lane, acc, 1 + a, ca, cb, single, status);
        break;
    }
  }
}

// The dense part of one tile, for one warp: the first step over all its rows
// (kGid: the step adds group-id contributions), then its survivors appended
// to the warp's list after the first n entries; returns the list length.
template <bool kHost, bool kText, bool kGid, bool kStaged = false>
__device__ __forceinline__ uint32_t tile_first_step(const DevQuery& Q, const PageState& P, const TileHdr& H,
                                                    uint32_t i0, uint32_t nmb, uint32_t row_base, const uint8_t* stab,
                                                    uint32_t* list, uint32_t n, int lane, unsigned int* status,
                                                    StagedPay sp = StagedPay{nullptr, 0, 0}) {
  TileState T;
  tile_init<kGid>(P, i0, nmb, lane, T);
  tile_dense_step<kHost, kText, kGid, kStaged>(Q, 0, P, H, T, stab, lane, status, sp);
  return tile_compact<kGid>(T, list, n, row_base, lane);
}

// The first step's column of Q in page P: its page address and packed words.
struct FirstCol {
  int c;
  uint32_t codec;
  const uint8_t* pg;
  const uint8_t* pay;
};
__device__ __forceinline__ FirstCol first_col(const DevQuery& Q, const PageState& P) {
  FirstCol f;
  f.c = Q.steps[0].col;
  f.codec = Q.cols[f.c].codec;
  f.pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, f.c));
  f.pay = f.pg + payload_offset(f.codec, P.prow);
  return f;
}

// One ticket: the rows [chunk*chunk_rows, +chunk_rows) of Q's fact table
// (a smaller range for the launch's last tickets: tail_first / tail_rows),
// processed by one warp, cut at page boundaries into tiles.  A page whose
// zone map misses the first step's value range is skipped whole; inside a
// page, mini blocks whose headers miss it are skipped by the first step.
// Each tile loads its headers as it starts (the other resident warps hide
// the latency).  The list collects the survivors of consecutive tiles (a
// segment of at most 2^kRowBits rows of one page) before the later steps and
// the aggregation run on them.
template <bool kHost, bool kText, bool kStage>
__device__ void process_ticket(const DevQuery& Q, uint64_t chunk, unsigned long long* acc, const uint8_t* stab,
                               uint32_t* list, int lane, unsigned int* status,
                               uint8_t* ring) {
  const uint64_t PR = Q.page_rows;
  uint64_t r0 = chunk * Q.chunk_rows, r1 = r0 + Q.chunk_rows;
  if (Q.tail_rows != 0 && chunk >= Q.tail_first) {  // one of the launch's small last tickets
    r0 = Q.tail_first * Q.chunk_rows + (chunk - Q.tail_first) * Q.tail_rows;
    r1 = r0 + Q.tail_rows;
  }
  r1 = tmin<uint64_t>(Q.nrows, r1);
  const bool gid0 = Q.nsteps != 0 && step_adds_gid(Q.steps[0]);
  for (uint64_t p = r0 / PR; p <= (r1 - 1) / PR; ++p) {
    const uint64_t pr0 = tmax<uint64_t>(r0, p * PR), pr1 = tmin<uint64_t>(r1, (p + 1) * PR);
    const uint32_t mb0 = uint32_t((pr0 - p * PR) / kMB);
    const uint32_t mb1 = uint32_t((pr1 - p * PR + kMB - 1) / kMB);
    const uint32_t ntiles = (mb1 - mb0 + TB - 1) / TB;
    if (Q.nsteps != 0) {  // zone map: skip a page the first step's range misses
      const DevStep& S0 = Q.steps[0];
      const int2 z = __ldg(Q.cols[S0.col].zone + p);
      if (S0.zlo > S0.zhi || z.y < S0.zlo || z.x > S0.zhi) continue;
    }
    PageState P;
    page_begin<kHost>(Q, p, lane, P);
    // staged first step (StageRing in tile.cuh): the headers of tiles 0 and 1
    // and the words of tile 0 are in flight before the first decode
    // a staged launch stages every query (the host makes it so)
    const uint32_t bwcap = kStage && !kHost ? Q.stage : 0u;
    if (kStage && bwcap == 0) {
      if (lane == 0) atomicOr(status, S_INTERNAL);
      return;
    }
    if (kStage) {
      const FirstCol f = first_col(Q, P);
      stage_headers(ring, 0, f.pg, f.codec, mb0, tmin<uint32_t>(TB, mb1 - mb0), lane);
      cp_async_commit();
      cp_async_wait_all();
      __syncwarp();
      stage_payload(ring, bwcap, 0, 0, f.pay, f.codec, mb0, tmin<uint32_t>(TB, mb1 - mb0), lane);
      if (ntiles > 1) stage_headers(ring, 1, f.pg, f.codec, mb0 + TB, tmin<uint32_t>(TB, mb1 - mb0 - TB), lane);
      cp_async_commit();
    }
    uint32_t n = 0, seg_mb = mb0;
    for (uint32_t j = 0; j < ntiles; ++j) {
      const uint32_t i0 = mb0 + j * TB;
      const uint32_t nmb = tmin<uint32_t>(TB, mb1 - i0);
      const uint32_t row_base = (i0 - seg_mb) * kMB;
      if constexpr (kStage) {
        cp_async_wait_all();  // this tile's words and the next tile's headers have landed
        __syncwarp();
        const FirstCol f = first_col(Q, P);
        if (j + 1 < ntiles)
          stage_payload(ring, bwcap, (j + 1) % 3, (j + 1) % 2, f.pay, f.codec, i0 + TB,
                        tmin<uint32_t>(TB, mb1 - i0 - TB), lane);
        if (j + 2 < ntiles) {
          const uint32_t n2 = tmin<uint32_t>(TB, mb1 - i0 - 2 * TB);
          stage_headers(ring, (j + 2) % 3, f.pg, f.codec, i0 + 2 * TB, n2, lane);
          prefetch_other_headers(Q, P, f.c, i0 + 2 * TB, n2, lane);
        }
        cp_async_commit();
        const TileHdr H = staged_headers(ring, j % 3, f.c, f.codec, i0, nmb, lane);
        const StagedPay sp{stage_words(ring, j % 2, bwcap), stage_pw(bwcap), bwcap};
        if (gid0) n = tile_first_step<kHost, kText, true, true>(Q, P, H, i0, nmb, row_base, stab, list, n, lane, status, sp);
        else n = tile_first_step<kHost, kText, false, true>(Q, P, H, i0, nmb, row_base, stab, list, n, lane, status, sp);
      } else {
        const TileHdr H = load_headers<kHost>(Q, P, i0, nmb, lane);
        if (!kHost && Q.pf_step) prefetch_words(Q, P, H, Q.steps[1].col, nmb, lane);
        if (gid0) n = tile_first_step<kHost, kText, true>(Q, P, H, i0, nmb, row_base, stab, list, n, lane, status);
        else n = tile_first_step<kHost, kText, false>(Q, P, H, i0, nmb, row_base, stab, list, n, lane, status);
      }
      const uint32_t next = i0 + TB;
      if (j + 1 == ntiles || n + kTileRows > kListCap || next + TB - seg_mb > kSegMbs) {
        n = list_steps<kHost, kText>(Q, P, seg_mb, list, n, stab, lane, status, 1);
        if (n) list_aggregate<kHost>(Q, P, seg_mb, list, n, lane, acc, status);
        n = 0;
        seg_mb = next;
      }
    }
  }
}

// Copies a query's shared-memory join tables into the CTA's table region:
// open-addressing slots as they are, direct tables as 1/2/4-byte group-id
// contributions (all ones = absent); builds the code-level matcher tables
// of string steps on FSST columns.
__device__ void load_smem_tables(const DevQuery& Q, uint8_t* stab) {
  for (uint32_t s = 0; s < Q.nsteps; ++s) {
    const DevStep& S = Q.steps[s];
    if ((S.kind == ST_PREFIX || S.kind == ST_CONTAINS) && S.smem_width != 0 && Q.cols[S.col].codec == C_FSST) {
      build_fsst_matcher(S, Q.cols[S.col].sym, Q.cols[S.col].nsym, stab + S.smem_off);
      continue;
    }
    if (S.kind != ST_PROBE || S.smem_width == 0) continue;
    if (S.ht_kind == HT_OPEN) {
      const uint2* src = static_cast<const uint2*>(S.ht);
      uint2* dst = reinterpret_cast<uint2*>(stab + S.smem_off);
      for (uint32_t i = threadIdx.x; i <= S.ht_mask; i += blockDim.x) dst[i] = __ldg(src + i);
      continue;
    }
    const uint32_t* src = static_cast<const uint32_t*>(S.ht);
    for (uint32_t i = threadIdx.x; i < S.krange; i += blockDim.x) {
      const uint32_t e = __ldg(src + i);
      const uint32_t c = (e & 0xffffu) * S.mul0 + (e >> 16) * S.mul1;
      if (S.smem_width == 1) stab[S.smem_off + i] = e == kAbsent ? 0xffu : uint8_t(c);
      else if (S.smem_width == 2)
        reinterpret_cast<uint16_t*>(stab + S.smem_off)[i] = e == kAbsent ? 0xffffu : uint16_t(c);
      else reinterpret_cast<uint32_t*>(stab + S.smem_off)[i] = e == kAbsent ? kAbsent : c;
    }
  }
}

// kText = false: the build without the general string matcher (CONTAINS,
// FSST), launched for batches that have no such step.  kStage: the build
// with the staging ring (device-resident batches without such steps,
// launched when the tuning asks for staging).  kThreads: the largest CTA
// the build launches with (512- and 1,024-thread CTAs, 2 and 1 per SM, keep
// the 64 registers of the 4 x 256-thread build).
template <bool kHost, int kMinBlocks, bool kText, bool kStage = false, int kThreads = 256>
__global__ void __launch_bounds__(kThreads, kMinBlocks) fused_kernel(const DevQuery* __restrict__ queries,
                                                       const uint64_t* __restrict__ qbegin, int nq,
                                                       uint64_t total, Sched* sched, uint32_t acc_slots,
                                                     uint32_t tables_bytes, uint32_t stage_bw) {
  extern __shared__ __align__(16) uint8_t dyn[];
  __shared__ CtaState cs;
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(dyn);
  uint8_t* stab = dyn + ((acc_slots * sizeof(unsigned long long) + 15) & ~size_t(15));
  uint32_t* lists = reinterpret_cast<uint32_t*>(stab + tables_bytes);
  // Warps draw tickets on their own (one ticket = chunk_rows rows of one
  // query, processed by one warp), so no CTA barrier separates tickets.  The
  // CTA meets only when its warps' tickets leave the current query: it then
  // moves to the smallest query any warp holds (tickets are handed out in
  // query order, so every warp reaches that meeting point), flushing the
  // finished query's accumulators first.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t* list = lists + uint32_t(warp) * kListCap;
  uint8_t* ring = reinterpret_cast<uint8_t*>(lists + nw * kListCap) + size_t(warp) * stage_warp_bytes(stage_bw);
  auto draw = [&](unsigned long long& t) -> int {
    unsigned long long x = 0;
    if (lane == 0) x = atomicAdd(&sched->next, 1ull);
    t = __shfl_sync(kFull, x, 0);
    if (t >= total) return INT_MAX;
    int lo = 0, hi = nq - 1;  // last query with qbegin <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (__ldg(qbegin + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  unsigned long long held;
  int hq = draw(held);
  int cur = -1;
  for (;;) {
    if (lane == 0) cs.wq[warp] = hq;
    __syncthreads();
    int next = INT_MAX;
    for (int w = 0; w < nw; ++w) next = min(next, cs.wq[w]);
    if (cur >= 0) finish_query(cs.q, sacc, cs.mine, cs);
    if (next == INT_MAX) break;
    {  // bring the query's plan into shared memory
      const uint4* src = reinterpret_cast<const uint4*>(queries + next);
      uint4* dst = reinterpret_cast<uint4*>(&cs.q);
      for (uint32_t i = threadIdx.x; i < sizeof(DevQuery) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    if (threadIdx.x == 0) cs.mine = 0;
    __syncthreads();
    const DevQuery& Q = cs.q;
    if (Q.use_smem_acc) {
      const uint32_t n = Q.domain * (1 + Q.naggs);
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sacc[i] = 0ull;
    }
    load_smem_tables(Q, stab);
    __syncthreads();
    cur = next;
    unsigned long long* acc = Q.use_smem_acc ? sacc : Q.acc;
    uint32_t done_here = 0;
    while (hq == cur) {
      process_ticket<kHost, kText, kStage>(Q, held - Q.chunk_begin, acc, stab, list, lane, &sched->status,
                                           ring);
      ++done_here;
      hq = draw(held);
    }
    if (lane == 0 && done_here) atomicAdd(&cs.mine, done_here);
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


template <bool kHost, int kMinBlocks, bool kText, bool kStage = false, int kThreads = 256>
int occupancy_of(int threads, size_t smem) {
  int n = 0;
  auto* k = fused_kernel<kHost, kMinBlocks, kText, kStage, kThreads>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
  return n;
}

template <bool kHost, int kMinBlocks, bool kText, bool kStage = false, int kThreads = 256>
cudaError_t launch_as(const FusedLaunch& L, size_t smem, uint32_t tb, cudaStream_t s) {
  auto* k = fused_kernel<kHost, kMinBlocks, kText, kStage, kThreads>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, smem, s>>>(
      L.queries, L.qbegin, L.nq, L.total_chunks, L.sched, L.acc_slots, tb, L.stage_bw);
  return cudaGetLastError();
}

}  // namespace
}  // namespace dpf

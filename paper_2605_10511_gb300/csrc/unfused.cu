// Unfused per-operator chain: the baseline the fused kernel is compared with.
//
// The same compiled plan runs as one kernel per operator, each writing its
// output to global memory for the next (the separate-kernel data path the
// paper measures DPF against, Sec. 5.1 "GiDP"): every referenced column is
// decoded into an int32 array (strings: lengths + absolute offsets), each
// predicate writes a flag array, a compaction turns flags into a row-id
// list, each join probes the list and compacts the hits into a new list,
// group keys are gathered, and an aggregation kernel adds int64 sums per
// group.  Row counts stay on the device, so the chain needs no host
// synchronisation and can be captured in a CUDA graph.
#include "../../include/dpf.h"
#include "dpf_device.cuh"
#include "kernels.h"

namespace dpf {
namespace {

__device__ __forceinline__ uint32_t page_mbs(uint64_t nrows, uint32_t P, uint64_t p) {
  const uint64_t rows = tmin<uint64_t>(P, nrows - p * P);
  return uint32_t((rows + kMB - 1) / kMB);
}

// One warp per mini block: header + payload -> 128 values written out.
__global__ void decode_col_kernel(DevColumn C, int32_t* out) {
  const int lane = threadIdx.x & 31;
  const uint64_t mbp = C.page_rows / kMB;
  const uint64_t npages = (C.nrows + C.page_rows - 1) / C.page_rows;
  const uint64_t total = npages * mbp;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t g = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; g < total; g += nw) {
    const uint64_t p = g / mbp;
    const uint32_t i = uint32_t(g % mbp);
    if (i >= page_mbs(C.nrows, C.page_rows, p)) continue;
    const uint32_t prow = uint32_t(tmin<uint64_t>(C.page_rows, C.nrows - p * C.page_rows));
    const uint8_t* pg = C.blob + __ldg(C.page_off + p);
    uint4 hv = make_uint4(0, 0, 0, 0);
    if (C.codec == C_DELTA) {
      hv = __ldg(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(i) * 16));
    } else {
      const uint2 h = __ldg(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(i) * 8));
      hv.x = h.x;
      hv.y = h.y;
    }
    const MbHdr H = parse_hdr(hv, C.codec);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(C.codec, prow)) + H.woff;
    uint32_t w[4], v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = (uint32_t(lane) < H.bw && H.bw <= 32) ? __ldg(pay + k * H.bw + lane) : 0u;
    decode_mb(w, H, C.codec, lane, v);
    const uint64_t r0 = p * C.page_rows + uint64_t(i) * kMB;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t j = k * 32 + lane;
      if (i * kMB + j < prow) out[r0 + j] = int32_t(v[k]);
    }
  }
}

// Strings: lengths and absolute byte offsets (within the column blob).
__global__ void decode_str_kernel(DevColumn C, int32_t* len_out, uint64_t* off_out) {
  const int lane = threadIdx.x & 31;
  const uint64_t mbp = C.page_rows / kMB;
  const uint64_t npages = (C.nrows + C.page_rows - 1) / C.page_rows;
  const uint64_t total = npages * mbp;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t g = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; g < total; g += nw) {
    const uint64_t p = g / mbp;
    const uint32_t i = uint32_t(g % mbp);
    const uint32_t nmb = page_mbs(C.nrows, C.page_rows, p);
    if (i >= nmb) continue;
    const uint32_t prow = uint32_t(tmin<uint64_t>(C.page_rows, C.nrows - p * C.page_rows));
    const uint64_t pbase = __ldg(C.page_off + p);
    const uint8_t* pg = C.blob + pbase;
    const uint2 h = __ldg(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(i) * 8));
    const uint32_t start = __ldg(reinterpret_cast<const uint32_t*>(pg + kPageHdr + uint64_t(nmb) * 8 + uint64_t(i) * 4));
    const uint32_t extra = __ldg(reinterpret_cast<const uint32_t*>(pg + 12));
    const MbHdr H = parse_hdr(make_uint4(h.x, h.y, 0, 0), C_STR);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(C_STR, prow)) + H.woff;
    uint32_t w[4], v[4], st[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = (uint32_t(lane) < H.bw && H.bw <= 32) ? __ldg(pay + k * H.bw + lane) : 0u;
    decode_mb(w, H, C_STR, lane, v);
    excl_scan128(v, lane, st);
    const uint64_t r0 = p * C.page_rows + uint64_t(i) * kMB;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t j = k * 32 + lane;
      if (i * kMB + j < prow) {
        len_out[r0 + j] = int32_t(v[k]);
        off_out[r0 + j] = pbase + extra + start + st[k];
      }
    }
  }
}

__global__ void pred_kernel(const int32_t* vals, uint64_t n, DevStep S, uint8_t* flags, int first) {
  for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += uint64_t(gridDim.x) * blockDim.x) {
    const uint8_t ok = step_pred(S, vals[r]) ? 1 : 0;
    flags[r] = first ? ok : uint8_t(flags[r] & ok);
  }
}

__global__ void prefix_kernel(const int32_t* len, const uint64_t* off, const uint8_t* blob, uint64_t n,
                              DevStep S, uint8_t* flags, int first) {
  for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += uint64_t(gridDim.x) * blockDim.x) {
    bool ok = uint32_t(len[r]) >= S.plen;
    for (uint32_t i = 0; ok && i < S.plen; ++i) ok = __ldg(blob + off[r] + i) == S.pfx[i];
    flags[r] = first ? uint8_t(ok) : uint8_t(flags[r] & uint8_t(ok));
  }
}

// Warp-aggregated append of (rid, gid) pairs to a list.
__device__ __forceinline__ void append(bool keep, uint32_t rid, uint32_t gid, uint32_t* rid_out,
                                       uint32_t* gid_out, unsigned long long* n_out) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(kFull, keep);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(n_out, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, __ffs(m) - 1);
  if (keep) {
    const uint64_t at = base + __popc(m & ((1u << lane) - 1u));
    rid_out[at] = rid;
    gid_out[at] = gid;
  }
}

__global__ void compact_kernel(const uint8_t* flags, uint64_t n, uint32_t* rid, uint32_t* gid,
                               unsigned long long* count) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t n_pad = (n + 31) & ~uint64_t(31);
  for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n_pad; r += stride) {
    const bool keep = r < n && flags[r];
    append(keep, uint32_t(r), 0u, rid, gid, count);
  }
}

__global__ void probe_kernel(const uint32_t* rid_in, const uint32_t* gid_in, const unsigned long long* n_in,
                             const int32_t* fk, DevStep S, uint32_t* rid_out, uint32_t* gid_out,
                             unsigned long long* n_out, unsigned int* status) {
  const uint64_t n = *n_in;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t n_pad = (n + 31) & ~uint64_t(31);
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
    bool hit = false;
    uint32_t r = 0, g = 0, pay = 0;
    if (i < n) {
      r = rid_in[i];
      g = gid_in[i];
      const int32_t key = fk[r];
      if (S.ht_kind == HT_DIRECT || S.ht_kind == HT_RANK) {
        const uint32_t off = uint32_t(key) - uint32_t(S.kmin);
        if (off < S.krange) {
          pay = S.ht_kind == HT_RANK ? rank_entry(S.ht, S.krange, off) : __ldg(static_cast<const uint32_t*>(S.ht) + off);
          hit = pay != kAbsent;
        }
      } else if (key != kEmptyKey) {
        hit = ht_probe(static_cast<const uint2*>(S.ht), S.ht_mask, key, &pay, status);
      }
    }
    append(hit, r, g + (pay & 0xffffu) * S.mul0 + (pay >> 16) * S.mul1, rid_out, gid_out, n_out);
  }
}

__global__ void key_kernel(const uint32_t* rid, uint32_t* gid, const unsigned long long* n_in, const int32_t* codes,
                           uint32_t mul) {
  const uint64_t n = *n_in;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    gid[i] += uint32_t(codes[rid[i]]) * mul;
}

struct AggArgs {
  const int32_t* a[4];
  const int32_t* b[4];
  uint32_t op[4];
  uint32_t naggs, domain;
  unsigned long long* acc;
  int smem;
};

__global__ void agg_kernel(const uint32_t* rid, const uint32_t* gid, const unsigned long long* n_in, AggArgs A,
                           unsigned int* status) {
  extern __shared__ unsigned long long sacc[];
  const uint32_t S1 = 1 + A.naggs;
  const uint32_t slots = A.domain * S1;
  if (A.smem) {
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) sacc[i] = 0ull;
    __syncthreads();
  }
  unsigned long long* acc = A.smem ? sacc : A.acc;
  const uint64_t n = *n_in;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t g = gid[i], r = rid[i];
    if (g >= A.domain) {
      atomicOr(status, S_CORRUPT);
      continue;
    }
    atomicAdd(acc + uint64_t(g) * S1, 1ull);
    for (uint32_t a = 0; a < A.naggs; ++a) {
      long long x;
      if (A.op[a] == DPF_AGG_COUNT) x = 1;
      else if (A.op[a] == DPF_AGG_SUM) x = A.a[a][r];
      else if (A.op[a] == DPF_AGG_SUM_MUL)
        x = (long long)((unsigned long long)(long long)A.a[a][r] * (unsigned long long)(long long)A.b[a][r]);
      else x = (long long)A.a[a][r] - (long long)A.b[a][r];
      atomicAdd(acc + uint64_t(g) * S1 + 1 + a, (unsigned long long)x);
    }
  }
  if (A.smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x)
      if (sacc[i]) atomicAdd(A.acc + i, sacc[i]);
  }
}

// Non-empty groups -> records in key order; clears the accumulators.
__global__ void assemble_kernel(const DevQuery* qd) {
  __shared__ unsigned int warp_sum[32];
  const DevQuery& Q = *qd;
  const uint32_t S1 = 1 + Q.naggs;
  dpf_record* out = reinterpret_cast<dpf_record*>(Q.out);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (Q.nkeys == 0) {
    if (threadIdx.x == 0) {
      dpf_record r;
      r.key[0] = r.key[1] = 0;
      r.count = (long long)Q.acc[0];
      for (int a = 0; a < 4; ++a) r.val[a] = a < int(Q.naggs) ? (long long)Q.acc[1 + a] : 0;
      out[0] = r;
      *Q.out_n = 1;
    }
  } else {
    uint32_t base = 0;
    for (uint32_t g0 = 0; g0 < Q.domain; g0 += blockDim.x) {
      const uint32_t g = g0 + threadIdx.x;
      const unsigned long long cnt = g < Q.domain ? Q.acc[uint64_t(g) * S1] : 0ull;
      const unsigned b = __ballot_sync(kFull, cnt != 0);
      if (lane == 0) warp_sum[warp] = __popc(b);
      __syncthreads();
      uint32_t before = 0, all = 0;
      for (int w2 = 0; w2 < nw; ++w2) {
        if (w2 < warp) before += warp_sum[w2];
        all += warp_sum[w2];
      }
      __syncthreads();
      if (cnt != 0) {
        dpf_record r;
        for (int k = 0; k < 2; ++k)
          r.key[k] = k < int(Q.nkeys) ? Q.key_dict[k][(g / Q.key_div[k]) % Q.key_dom[k]] : 0;
        r.count = (long long)cnt;
        for (int a = 0; a < 4; ++a) r.val[a] = a < int(Q.naggs) ? (long long)Q.acc[uint64_t(g) * S1 + 1 + a] : 0;
        out[base + before + __popc(b & ((1u << lane) - 1u))] = r;
      }
      base += all;
    }
    if (threadIdx.x == 0) *Q.out_n = base;
  }
  __syncthreads();
  for (uint64_t i = threadIdx.x; i < uint64_t(Q.domain) * S1; i += blockDim.x) Q.acc[i] = 0ull;
}

int grid_for(uint64_t n, int threads) {
  return int(tmax<uint64_t>(1, tmin<uint64_t>((n + threads - 1) / threads, 152ull * 16)));
}

}  // namespace

cudaError_t launch_unfused(const UnfusedChain& U, cudaStream_t s, uint32_t* launches) {
  const DevQuery& Q = U.q;
  const uint64_t n = Q.nrows;
  uint32_t L = 0;
  cudaError_t e = cudaMemsetAsync(U.counts, 0, sizeof(unsigned long long) * kUnfusedCounts, s);
  if (e != cudaSuccess) return e;
  // 1. decode every referenced column
  for (uint32_t c = 0; c < Q.ncols; ++c) {
    const int g = grid_for((n + kMB - 1) / kMB * 32, 256);
    if (Q.cols[c].codec == C_STR) decode_str_kernel<<<g, 256, 0, s>>>(Q.cols[c], U.lens[c], U.offs[c]);
    else decode_col_kernel<<<g, 256, 0, s>>>(Q.cols[c], U.vals[c]);
    ++L;
  }
  // 2. predicates -> flags
  bool first = true;
  for (uint32_t i = 0; i < Q.nsteps; ++i) {
    const DevStep& S = Q.steps[i];
    if (S.kind == ST_PROBE || S.kind == ST_KEY) continue;
    const int g = grid_for(n, 256);
    if (S.kind == ST_PREFIX)
      prefix_kernel<<<g, 256, 0, s>>>(U.lens[S.col], U.offs[S.col], Q.cols[S.col].blob, n, S, U.flags, first);
    else
      pred_kernel<<<g, 256, 0, s>>>(U.vals[S.col], n, S, U.flags, first);
    first = false;
    ++L;
  }
  if (first) {
    e = cudaMemsetAsync(U.flags, 1, n, s);
    if (e != cudaSuccess) return e;
  }
  // 3. compaction -> row-id list
  compact_kernel<<<grid_for(n, 256), 256, 0, s>>>(U.flags, n, U.rid[0], U.gid[0], U.counts + 0);
  ++L;
  // 4. joins
  int cur = 0, slot = 1;
  for (uint32_t i = 0; i < Q.nsteps; ++i) {
    const DevStep& S = Q.steps[i];
    if (S.kind != ST_PROBE) continue;
    probe_kernel<<<grid_for(n, 256), 256, 0, s>>>(U.rid[cur], U.gid[cur], U.counts + slot - 1, U.vals[S.col], S,
                                                 U.rid[cur ^ 1], U.gid[cur ^ 1], U.counts + slot,
                                                 &U.sched->status);
    cur ^= 1;
    ++slot;
    ++L;
  }
  // 5. group keys from dictionary columns
  for (uint32_t i = 0; i < Q.nsteps; ++i) {
    const DevStep& S = Q.steps[i];
    if (S.kind != ST_KEY) continue;
    key_kernel<<<grid_for(n, 256), 256, 0, s>>>(U.rid[cur], U.gid[cur], U.counts + slot - 1, U.vals[S.col], S.key_mul);
    ++L;
  }
  // 6. aggregation
  AggArgs A{};
  A.naggs = Q.naggs;
  A.domain = Q.domain;
  A.acc = Q.acc;
  for (uint32_t a = 0; a < Q.naggs; ++a) {
    A.op[a] = Q.agg_op[a];
    A.a[a] = U.vals[Q.agg_a[a]];
    A.b[a] = U.vals[Q.agg_b[a]];
  }
  const uint64_t slots = uint64_t(Q.domain) * (1 + Q.naggs);
  A.smem = slots <= kSmemAccSlots ? 1 : 0;
  agg_kernel<<<grid_for(n, 256), 256, A.smem ? slots * 8 : 0, s>>>(U.rid[cur], U.gid[cur], U.counts + slot - 1, A,
                                                                 &U.sched->status);
  ++L;
  // 7. records
  assemble_kernel<<<1, 1024, 0, s>>>(U.dq);
  ++L;
  if (launches) *launches = L;
  return cudaGetLastError();
}

}  // namespace dpf

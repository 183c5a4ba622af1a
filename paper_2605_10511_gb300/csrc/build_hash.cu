// Table scan + hash build (Kernel #1 of Sec. 3.1: scan, filter, build) and
// scan + probe + build (Kernel #2: the scan also probes tables built
// earlier, so a chain of joins is built table by table).
//
// The table's columns are decoded tile by tile with the same warp tiles as
// the fused kernel, and its steps (predicates, then probes of earlier
// tables, all in global memory) run the same dense first step and survivor
// list code.  Rows that pass are either counted (first pass, sizes the
// table) or inserted (second pass) into an open-addressing table with
// linear probing or a direct table.  An open slot is one 64-bit word
// {key, payload} claimed with a single compare-and-swap; the payload packs
// two 16-bit fields.
//
// Payload field f comes from Q.build_pay[f]: a value >= kPayFromGid holds
// {shift << 8 | bits}, and the field is bits [shift, shift + bits) of the
// row's group id, which the scan's steps built (a probe step adds its
// match's payload fields times their multipliers, a key step a DICT code
// times its multiplier: the fused kernel's group-id machinery carries the
// fields through the survivor list); another value >= 0 is the index of a
// DICT column of the scanned table (the field is its code); a value < 0
// encodes code = -1 - build_pay[f], and the field is payload field
// (code & 1) of the row's match in the table probed by step (code >> 1).
#include "build_pay.h"
#include "tile.cuh"

namespace dpf {
namespace {

// Payload field f of a kept row (warp-uniform call; lanes with !valid
// return 0).  A probe step's match is looked up again here; the row passed
// that step, so a miss means a corrupt table and sets S_INTERNAL.
template <bool kHost>
__device__ __forceinline__ uint32_t build_payload(const DevQuery& Q, int f, const PageState& P, uint32_t i0,
                                                  uint32_t r, uint32_t gid, bool valid, int lane,
                                                  unsigned int* status) {
  const int32_t src = Q.build_pay[f];
  if (src >= kPayFromGid) {
    const uint32_t sh = (uint32_t(src) >> 8) & 0xffu, bits = uint32_t(src) & 0xffu;
    return valid ? (gid >> sh) & ((1u << bits) - 1u) : 0u;
  }
  if (src >= 0) return row_value<kHost>(Q, src, P, i0, r, valid, lane, status);
  const uint32_t code = uint32_t(-1 - src);
  const DevStep& S = Q.steps[code >> 1];
  const uint32_t key = row_value<kHost>(Q, S.col, P, i0, r, valid, lane, status);
  if (!valid) return 0u;
  uint32_t pay = 0;
  bool hit;
  if (S.ht_kind == HT_DIRECT || S.ht_kind == HT_RANK) {
    const uint32_t off = key - uint32_t(S.kmin);
    pay = off >= S.krange ? kAbsent
          : S.ht_kind == HT_RANK ? rank_entry(S.ht, S.krange, off)
                                 : __ldg(static_cast<const uint32_t*>(S.ht) + off);
    hit = pay != kAbsent;
  } else {
    hit = int32_t(key) != kEmptyKey && ht_probe(static_cast<const uint2*>(S.ht), S.ht_mask, int32_t(key), &pay, status);
  }
  if (!hit) {
    atomicOr(status, S_INTERNAL);
    return 0u;
  }
  return (code & 1u) ? pay >> 16 : pay & 0xffffu;
}

constexpr unsigned long long kEmptySlot = 0x0000000080000000ull;  // {INT32_MIN, 0}

// kMode 0: count kept rows and their key range; 1: insert into an
// open-addressing table; 2: insert into a direct table; 3: set the rows'
// presence bits of a rank directory (a bit already set is a duplicate key)
// and write {key offset, payload} to the staging list (a tile reserves one
// slot per kept row with one atomic), from which rank_scatter places the
// payloads once the ranks are known.  Modes 1-3
// also add the rows they insert to L.inserted when it is set (a table sized
// before its scan learns its entry count that way).
template <bool kHost, int kMode>
__global__ void __launch_bounds__(256) build_kernel(const DevQuery* __restrict__ qdev, BuildLaunch L,
                                                    unsigned int* status) {
  __shared__ __align__(16) DevQuery Q;
  __shared__ uint32_t lists[8 * kTileRows];
  {
    const uint4* src = reinterpret_cast<const uint4*>(qdev);
    uint4* dst = reinterpret_cast<uint4*>(&Q);
    for (uint32_t i = threadIdx.x; i < sizeof(DevQuery) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t* list = lists + (threadIdx.x >> 5) * kTileRows;
  const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const uint64_t PR = Q.page_rows;
  const uint64_t npages = (Q.nrows + PR - 1) / PR;
  const uint64_t tiles_per_page = (PR / kMB + TB - 1) / TB;
  unsigned long long kept = 0;
  int32_t kmin = INT32_MAX, kmax = INT32_MIN;
  for (uint64_t w = warp; w < npages * tiles_per_page; w += nwarps) {
    const uint64_t p = w / tiles_per_page;
    const uint32_t i0 = uint32_t(w % tiles_per_page) * TB;
    PageState P;
    page_begin<kHost>(Q, p, lane, P);
    if (i0 >= P.nmb_page) continue;
    const uint32_t nmb = tmin<uint32_t>(TB, P.nmb_page - i0);
    const TileHdr H = load_headers<kHost>(Q, P, i0, nmb, lane);
    TileState T;
    tile_init(P, i0, nmb, lane, T);
    tile_dense_step<kHost>(Q, 0, P, H, T, nullptr, lane, status);
    uint32_t n = tile_compact(T, list, 0, 0, lane);
    n = list_steps<kHost>(Q, P, i0, list, n, nullptr, lane, status);
    // rank builds: one staging slot per kept row of the tile, reserved at once
    unsigned long long sbase = 0;
    if (kMode == 3 && n != 0) {
      if (lane == 0) sbase = atomicAdd(L.stage_n, (unsigned long long)n);
      sbase = __shfl_sync(kFull, sbase, 0);
    }
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
      const bool valid = j0 + lane < n;
      const uint32_t e = valid ? list[j0 + lane] : 0u;
      const uint32_t r = e & ((1u << kRowBits) - 1u), gid = e >> kRowBits;
      const int32_t kv = int32_t(row_value<kHost>(Q, Q.build_key, P, i0, r, valid, lane, status));
      const uint32_t c0 =
          kMode != 0 && Q.build_npay > 0 ? build_payload<kHost>(Q, 0, P, i0, r, gid, valid, lane, status) : 0u;
      const uint32_t c1 =
          kMode != 0 && Q.build_npay > 1 ? build_payload<kHost>(Q, 1, P, i0, r, gid, valid, lane, status) : 0u;
      if (!valid) continue;
      if (kMode == 0) {
        ++kept;
        kmin = min(kmin, kv);
        kmax = max(kmax, kv);
        continue;
      }
      // a rank build's slot of a row that inserts nothing holds a pair the
      // scatter skips (its key offset is out of range)
      const unsigned long long sslot = sbase + j0 + lane;
      if (kv == kEmptyKey) {
        atomicOr(status, S_CORRUPT);
        if (kMode == 3 && sslot < L.rank_cap) L.rank_stage[sslot] = make_uint2(0xffffffffu, 0u);
        continue;
      }
      ++kept;  // rows inserted (read only when L.inserted is set)
      const uint32_t pay = (c0 & 0xffffu) | ((c1 & 0xffffu) << 16);
      if (kMode == 2 || kMode == 3) {
        const uint32_t off = uint32_t(kv) - uint32_t(L.kmin);
        if (off >= L.krange) {
          atomicOr(status, S_INTERNAL);
          if (kMode == 3 && sslot < L.rank_cap) L.rank_stage[sslot] = make_uint2(0xffffffffu, 0u);
          continue;
        }
        if (kMode == 2) {
          if (atomicCAS(L.direct + off, kAbsent, pay) != kAbsent) atomicOr(status, S_DUPKEY);
        } else {
          unsigned int* word = reinterpret_cast<unsigned int*>(L.rank_dir + (off >> 6)) + ((off >> 5) & 1u);
          const unsigned int bit = 1u << (off & 31u);
          if (atomicOr(word, bit) & bit) atomicOr(status, S_DUPKEY);
          if (sslot < L.rank_cap) L.rank_stage[sslot] = make_uint2(off, pay);
          else atomicOr(status, S_INTERNAL);
        }
        continue;
      }
      const unsigned long long slot = (unsigned long long)uint32_t(kv) | ((unsigned long long)pay << 32);
      uint32_t h = fmix32(uint32_t(kv)) & L.mask;
      bool done = false;
      for (uint32_t q = 0; q <= L.mask && !done; ++q) {
        unsigned long long* addr = reinterpret_cast<unsigned long long*>(L.table + h);
        const unsigned long long old = atomicCAS(addr, kEmptySlot, slot);
        if (old == kEmptySlot) {
          done = true;
        } else if (int32_t(uint32_t(old)) == kv) {
          atomicOr(status, S_DUPKEY);
          done = true;
        } else {
          h = (h + 1) & L.mask;
        }
      }
      if (!done) atomicOr(status, S_INTERNAL);
    }
    __syncwarp();
  }
  if (kMode == 0) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      kept += __shfl_down_sync(kFull, kept, d);
      kmin = min(kmin, __shfl_down_sync(kFull, kmin, d));
      kmax = max(kmax, __shfl_down_sync(kFull, kmax, d));
    }
    if (lane == 0 && kept) {
      atomicAdd(L.count, kept);
      atomicMin(L.kminmax, kmin);
      atomicMax(L.kminmax + 1, kmax);
    }
  } else if (L.inserted) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) kept += __shfl_down_sync(kFull, kept, d);
    if (lane == 0 && kept) atomicAdd(L.inserted, kept);
  }
}

// Ranks of a rank directory: word w's counts = the present keys in words
// < w (z), and that plus the word's keys 0-31 (w).
// Pass 1: per block of 1,024 words, their total; pass 2 (one block): the
// exclusive prefix of the block totals; pass 3: each block's words.
constexpr uint32_t kRankBlockWords = 1024;
__device__ __forceinline__ uint32_t word_bits(const uint4& d) { return uint32_t(__popc(d.x) + __popc(d.y)); }

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* total) {
  __shared__ uint32_t warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) before += warp_tot[w];
    all += warp_tot[w];
  }
  __syncthreads();
  *total = all;
  return before + incl - x;
}

__global__ void rank_block_sums(const uint4* dir, uint32_t nwords, uint32_t* sums) {
  uint32_t x = 0;
  for (uint32_t k = 0; k < kRankBlockWords / 256; ++k) {
    const uint32_t w = blockIdx.x * kRankBlockWords + k * 256 + threadIdx.x;
    if (w < nwords) x += word_bits(dir[w]);
  }
  uint32_t total;
  block_excl_scan(x, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void rank_scan_sums(uint32_t* sums, uint32_t n) {
  uint32_t carry = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const uint32_t x = i < n ? sums[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan(x, &total);
    if (i < n) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void rank_fill(uint4* dir, uint32_t nwords, const uint32_t* sums) {
  uint32_t carry = sums[blockIdx.x];
  for (uint32_t k = 0; k < kRankBlockWords / 256; ++k) {
    const uint32_t w = blockIdx.x * kRankBlockWords + k * 256 + threadIdx.x;
    uint4 d = w < nwords ? dir[w] : make_uint4(0, 0, 0, 0);
    uint32_t total;
    const uint32_t ex = block_excl_scan(w < nwords ? word_bits(d) : 0u, &total);
    if (w < nwords) {
      d.z = carry + ex;
      d.w = d.z + uint32_t(__popc(d.x));
      dir[w] = d;
    }
    carry += total;
  }
}

// Payloads of a rank table at their ranks: each staged {key offset,
// payload} goes to the word's running count plus the set bits below it
// (a pair whose offset is outside the key range marks a row that inserted
// nothing).
__global__ void rank_scatter(const uint4* dir, const uint2* stage, const unsigned long long* n, uint32_t* pay,
                             uint32_t cap, uint32_t krange, unsigned int* status) {
  const uint64_t cnt = tmin<uint64_t>(*n, cap);
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint2 e = stage[i];
    if (e.x >= krange) continue;
    const uint4 d = dir[e.x >> 6];
    const uint32_t b = e.x & 63u, bb = b & 31u;
    const uint32_t idx = (b < 32 ? d.z : d.w) + uint32_t(__popc((b < 32 ? d.x : d.y) & ((1u << bb) - 1u)));
    if (idx < cap) pay[idx] = e.y;
    else atomicOr(status, S_INTERNAL);
  }
}

__global__ void init_table_kernel(uint2* table, uint32_t slots) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x)
    reinterpret_cast<unsigned long long*>(table)[i] = kEmptySlot;
}

int build_grid(uint64_t nrows, uint64_t page_rows) {
  const uint64_t npages = (nrows + page_rows - 1) / page_rows;
  const uint64_t tiles = npages * ((page_rows / kMB + TB - 1) / TB);
  const uint64_t blocks = (tiles + 7) / 8;  // 8 warps per block
  return int(tmin<uint64_t>(tmax<uint64_t>(blocks, 1), 4096));
}

}  // namespace

template <int kMode>
cudaError_t launch_build_mode(const BuildLaunch& L, cudaStream_t s) {
  const int g = build_grid(L.nrows, L.page_rows);
  if (L.host_data) build_kernel<true, kMode><<<g, 256, 0, s>>>(L.q, L, &L.sched->status);
  else build_kernel<false, kMode><<<g, 256, 0, s>>>(L.q, L, &L.sched->status);
  return cudaGetLastError();
}

cudaError_t launch_build_count(const BuildLaunch& L, cudaStream_t s) { return launch_build_mode<0>(L, s); }

cudaError_t launch_build_insert(const BuildLaunch& L, cudaStream_t s) {
  if (L.rank_dir) {  // presence bits and staged pairs, ranks, then payloads at their ranks
    const uint32_t nwords = uint32_t((uint64_t(L.krange) + 63) >> 6);
    const uint32_t nblocks = (nwords + kRankBlockWords - 1) / kRankBlockWords;
    cudaError_t e = launch_build_mode<3>(L, s);
    if (e != cudaSuccess) return e;
    rank_block_sums<<<nblocks, 256, 0, s>>>(L.rank_dir, nwords, L.rank_sums);
    rank_scan_sums<<<1, 1024, 0, s>>>(L.rank_sums, nblocks);
    rank_fill<<<nblocks, 256, 0, s>>>(L.rank_dir, nwords, L.rank_sums);
    const int g = int(tmax<uint32_t>(1u, tmin<uint32_t>((L.rank_cap + 255) / 256, 2048u)));
    rank_scatter<<<g, 256, 0, s>>>(L.rank_dir, L.rank_stage, L.stage_n, L.rank_pay, L.rank_cap, L.krange,
                                   &L.sched->status);
    return cudaGetLastError();
  }
  return L.direct ? launch_build_mode<2>(L, s) : launch_build_mode<1>(L, s);
}

cudaError_t launch_init_table(uint2* table, uint32_t slots, cudaStream_t s) {
  const int g = int(tmin<uint32_t>((slots + 255) / 256, 2048u));
  init_table_kernel<<<g, 256, 0, s>>>(table, slots);
  return cudaGetLastError();
}

cudaError_t launch_init_direct(uint32_t* table, uint32_t n, cudaStream_t s) {
  return cudaMemsetAsync(table, 0xff, size_t(n) * 4, s);
}

}  // namespace dpf

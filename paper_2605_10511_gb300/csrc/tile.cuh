// Warp tiles: TB consecutive mini blocks of one page processed by one warp.
//
// A tile walks the compiled steps of a query (Sec. 3.2 operation stage) over
// its 128*TB rows: each step decodes one column for the mini blocks that
// still hold live rows (the decompression stage, Sec. 3.4.1 / 4.1), then
// applies a predicate, a hash probe or a group-key contribution.  Row state
// stays in registers: one live bit per row (bit 4t+k = row 32k+lane of mini
// block t, a per-lane slice of the warp's ballot selection vector) and the
// dense group id.  Mini blocks without a live row are neither loaded nor
// decoded for later columns.
#pragma once

#include "dpf_device.cuh"
#include "kernels.h"

namespace dpf {

constexpr int TB = int(kMbPerWarpTile);

struct TileState {
  uint32_t alive;         // bit 4t+k: row 32k+lane of mini block t is live
  uint32_t gid[TB][4];    // dense group id of each row
  uint4 hdr;              // lane L: header of (column L / TB, mini block L % TB)
  uint32_t sstart;        // lane L: STR byte start of that mini block
  uint64_t pg;            // lane c: address of column c's page
  uint32_t extra;         // lane c: STR byte-region offset of column c's page
  uint32_t prow;          // rows in the page
  uint32_t i0, nmb;       // first mini block (page-relative), mini blocks in the tile
};

// Loads page addresses and every column's headers for a tile.
template <bool kHost>
__device__ __forceinline__ void tile_begin(const DevQuery& Q, uint64_t page, uint32_t i0,
                                           uint32_t nmb, int lane, TileState& T) {
  T.prow = uint32_t(tmin<uint64_t>(Q.page_rows, Q.nrows - page * Q.page_rows));
  T.i0 = i0;
  T.nmb = nmb;
  const uint32_t nmb_page = (T.prow + kMB - 1) / kMB;
  T.pg = 0;
  T.extra = 0;
  if (lane < int(Q.ncols)) {
    const DevColumn& C = Q.cols[lane];
    T.pg = reinterpret_cast<uint64_t>(C.blob) + __ldg(C.page_off + page);
  }
  const int hc = lane / TB, ht = lane % TB;
  const uint64_t hpg = __shfl_sync(kFull, T.pg, hc < int(Q.ncols) ? hc : 0);
  T.hdr = make_uint4(0, 0, 0, 0);
  T.sstart = 0;
  if (hc < int(Q.ncols) && ht < int(nmb)) {
    const uint32_t codec = Q.cols[hc].codec;
    const uint8_t* pg = reinterpret_cast<const uint8_t*>(hpg);
    if (codec == C_DELTA) {
      T.hdr = ld_u4<kHost>(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(i0 + ht) * 16));
    } else {
      const uint2 h = ld_u2<kHost>(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(i0 + ht) * 8));
      T.hdr.x = h.x;
      T.hdr.y = h.y;
      if (codec == C_STR)
        T.sstart = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(
            pg + kPageHdr + uint64_t(nmb_page) * 8 + uint64_t(i0 + ht) * 4));
    }
  }
  if (lane < int(Q.ncols) && Q.cols[lane].codec == C_STR)
    T.extra = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(T.pg + 12));
  T.alive = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t r = (i0 + t) * kMB + k * 32 + lane;
      if (t < int(nmb) && r < T.prow) T.alive |= 1u << (4 * t + k);
      T.gid[t][k] = 0;
    }
}

// Loads and decodes column c for the mini blocks with live rows.
// anym bit t = mini block t was decoded.  H receives the headers.
template <bool kHost>
__device__ __forceinline__ void tile_decode(const DevQuery& Q, int c, const TileState& T, int lane,
                                            uint32_t (&v)[TB][4], uint32_t& anym,
                                            MbHdr (&H)[TB], unsigned int* status) {
  const uint32_t codec = Q.cols[c].codec;
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, T.pg, c));
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(codec, T.prow));
  uint32_t w[TB][4];
  anym = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    bool any = __any_sync(kFull, (T.alive >> (4 * t)) & 15u) != 0;
    uint4 hv;
    hv.x = __shfl_sync(kFull, T.hdr.x, c * TB + t);
    hv.y = __shfl_sync(kFull, T.hdr.y, c * TB + t);
    hv.z = __shfl_sync(kFull, T.hdr.z, c * TB + t);
    hv.w = 0;
    H[t] = parse_hdr(hv, codec);
    if (any && H[t].bw > 32) {
      if (lane == 0) atomicOr(status, S_CORRUPT);
      any = false;
    }
    anym |= uint32_t(any) << t;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[t][k] = (any && uint32_t(lane) < H[t].bw)
                    ? ld_u32<kHost>(pay + H[t].woff + uint32_t(k) * H[t].bw + lane)
                    : 0u;
  }
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if ((anym >> t) & 1u) decode_mb(w[t], H[t], codec, lane, v[t]);
    else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[t][k] = 0;
    }
  }
}

// PREFIX step over a STR column: lengths are decoded, their exclusive scan
// gives each string's start, and the first plen bytes are compared.
template <bool kHost>
__device__ __forceinline__ void tile_prefix(const DevQuery& Q, const DevStep& S, TileState& T,
                                            int lane, unsigned int* status) {
  uint32_t len[TB][4];
  uint32_t anym;
  MbHdr H[TB];
  tile_decode<kHost>(Q, S.col, T, lane, len, anym, H, status);
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, T.pg, S.col));
  const uint8_t* bytes = pg + __shfl_sync(kFull, T.extra, S.col);
  const uint32_t plen = S.plen;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t st[4];
    excl_scan128(len[t], lane, st);
    const uint32_t mb_start = __shfl_sync(kFull, T.sstart, S.col * TB + t);
    uint32_t match = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (((T.alive >> (4 * t + k)) & 1u) && len[t][k] >= plen) match |= 1u << k;
    for (uint32_t i = 0; i < plen; ++i) {
      if (!__any_sync(kFull, match)) break;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((match >> k) & 1u) {
          const uint8_t b = ld_u8<kHost>(bytes + uint64_t(mb_start) + st[k] + i);
          if (b != S.pfx[i]) match &= ~(1u << k);
        }
    }
    T.alive &= ~((~match & 15u) << (4 * t));
  }
}

// Hash probe step: live rows that miss are dropped; hits add the payload
// fields to the group id.
template <bool kHost>
__device__ __forceinline__ void tile_probe(const DevQuery& Q, const DevStep& S, TileState& T,
                                           const uint8_t* stab, int lane, unsigned int* status) {
  uint32_t v[TB][4];
  uint32_t anym;
  MbHdr H[TB];
  tile_decode<kHost>(Q, S.col, T, lane, v, anym, H, status);
  const bool in_smem = S.ht_smem >= 0;
  const uint2* tab = in_smem ? reinterpret_cast<const uint2*>(stab + Q.tables[S.ht_smem].offset) : S.ht;
  const uint32_t mask = S.ht_mask;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    // all four probes of the lane advance together
    uint32_t h[4], pend = 0, hit = 0, pay[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = fmix32(v[t][k]) & mask;
      pay[k] = 0;
      // the empty-slot sentinel is never a stored key
      if (((T.alive >> (4 * t + k)) & 1u) && int32_t(v[t][k]) != kEmptyKey) pend |= 1u << k;
    }
    for (uint32_t n = 0; pend && n <= mask; ++n) {
      uint2 s[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((pend >> k) & 1u) s[k] = in_smem ? tab[h[k]] : __ldg(tab + h[k]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((pend >> k) & 1u)) continue;
        if (s[k].x == v[t][k]) {
          hit |= 1u << k;
          pay[k] = s[k].y;
          pend &= ~(1u << k);
        } else if (int32_t(s[k].x) == kEmptyKey) {
          pend &= ~(1u << k);
        } else {
          h[k] = (h[k] + 1) & mask;
        }
      }
    }
    if (pend) atomicOr(status, S_INTERNAL);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      T.gid[t][k] += (pay[k] & 0xffffu) * S.mul0 + (pay[k] >> 16) * S.mul1;
    const uint32_t live = (T.alive >> (4 * t)) & 15u;
    T.alive &= ~((live & ~hit & 15u) << (4 * t));
  }
}

// Predicate (RANGE / NOTRANGE / IN / FALSE) or group-key step.
template <bool kHost>
__device__ __forceinline__ void tile_filter_or_key(const DevQuery& Q, const DevStep& S,
                                                   TileState& T, int lane, unsigned int* status) {
  uint32_t v[TB][4];
  uint32_t anym;
  MbHdr H[TB];
  tile_decode<kHost>(Q, S.col, T, lane, v, anym, H, status);
  if (S.kind == ST_KEY) {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) T.gid[t][k] += v[t][k] * S.key_mul;
    return;
  }
  uint32_t keep = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (step_pred(S, int32_t(v[t][k]))) keep |= 1u << (4 * t + k);
  T.alive &= keep;
}

// Runs every step of the query on a tile; returns false if no row survived.
template <bool kHost>
__device__ __forceinline__ bool tile_steps(const DevQuery& Q, TileState& T, const uint8_t* stab,
                                           int lane, unsigned int* status) {
  for (uint32_t s = 0; s < Q.nsteps; ++s) {
    if (!__any_sync(kFull, T.alive)) return false;
    const DevStep& S = Q.steps[s];
    if (S.kind == ST_PREFIX) tile_prefix<kHost>(Q, S, T, lane, status);
    else if (S.kind == ST_PROBE) tile_probe<kHost>(Q, S, T, stab, lane, status);
    else tile_filter_or_key<kHost>(Q, S, T, lane, status);
  }
  return __any_sync(kFull, T.alive) != 0;
}

}  // namespace dpf

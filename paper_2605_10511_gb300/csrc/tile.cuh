// Warp tiles: TB consecutive mini blocks of one page processed by one warp.
//
// A tile walks the compiled steps of a query (Sec. 3.2 operation stage) over
// its 128*TB rows: each step decodes one column for the mini blocks that
// still hold live rows (the decompression stage, Sec. 3.4.1 / 4.1), then
// applies a predicate, a join probe or a group-key contribution.  Row state
// stays in registers: one live bit per row (bit 4t+k = row 32k+lane of mini
// block t, the lane's slice of the warp's ballot selection vector) and the
// dense group id.  Mini blocks without a live row are neither loaded nor
// decoded for later columns.
#pragma once

#include "dpf_device.cuh"
#include "kernels.h"

namespace dpf {

constexpr int TB = int(kMbPerWarpTile);

// Per warp and page: lane c holds column c's page address and, for strings,
// the offset of the page's byte region.
struct PageState {
  uint64_t pg;
  uint32_t extra;
  uint32_t prow;       // rows in the page
  uint32_t nmb_page;   // mini blocks in the page
};

template <bool kHost>
__device__ __forceinline__ void page_begin(const DevQuery& Q, uint64_t page, int lane, PageState& P) {
  P.prow = uint32_t(tmin<uint64_t>(Q.page_rows, Q.nrows - page * Q.page_rows));
  P.nmb_page = (P.prow + kMB - 1) / kMB;
  P.pg = 0;
  P.extra = 0;
  if (lane < int(Q.ncols)) {
    const DevColumn& C = Q.cols[lane];
    P.pg = reinterpret_cast<uint64_t>(C.blob) + __ldg(C.page_off + page);
    if (C.codec == C_STR) P.extra = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(P.pg + 12));
  }
}

// Lane L holds the header of (column L / TB, mini block i0 + L % TB).
struct TileHdr {
  uint32_t x, y, z;   // FOR/DICT/STR: {base, wob}; DELTA: {first, dmin, wob}
  uint32_t sstart;    // STR: byte start of the mini block
};

template <bool kHost>
__device__ __forceinline__ TileHdr load_headers(const DevQuery& Q, const PageState& P, uint32_t i0,
                                                uint32_t nmb, int lane) {
  TileHdr h{0, 0, 0, 0};
  const int hc = lane / TB, ht = lane % TB;
  const uint64_t hpg = __shfl_sync(kFull, P.pg, hc < int(Q.ncols) ? hc : 0);
  if (hc < int(Q.ncols) && ht < int(nmb)) {
    const uint32_t codec = Q.cols[hc].codec;
    const uint8_t* pg = reinterpret_cast<const uint8_t*>(hpg);
    if (codec == C_DELTA) {
      const uint4 v = ld_u4<kHost>(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(i0 + ht) * 16));
      h.x = v.x;
      h.y = v.y;
      h.z = v.z;
    } else {
      const uint2 v = ld_u2<kHost>(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(i0 + ht) * 8));
      h.x = v.x;
      h.y = v.y;
      if (codec == C_STR)
        h.sstart = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(
            pg + kPageHdr + uint64_t(P.nmb_page) * 8 + uint64_t(i0 + ht) * 4));
    }
  }
  return h;
}

struct TileState {
  uint32_t alive;         // bit 4t+k: row 32k+lane of mini block t is live
  uint32_t gid[TB][4];    // dense group id of each row
};

__device__ __forceinline__ void tile_init(const PageState& P, uint32_t i0, uint32_t nmb, int lane,
                                          TileState& T) {
  T.alive = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t r = (i0 + t) * kMB + k * 32 + lane;
      if (t < int(nmb) && r < P.prow) T.alive |= 1u << (4 * t + k);
      T.gid[t][k] = 0;
    }
}

// Loads and decodes column c for the mini blocks with live rows: v[t][k]
// = value of row 32k + lane of mini block t (the payload words are loaded
// into v and decoded in place).  anym bit t = mini block t was decoded.
template <bool kHost>
__device__ __forceinline__ void tile_decode(const DevQuery& Q, int c, const PageState& P, const TileHdr& Hd,
                                            uint32_t alive, int lane, uint32_t (&v)[TB][4], uint32_t& anym,
                                            unsigned int* status) {
  const uint32_t codec = Q.cols[c].codec;
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(codec, P.prow));
  uint32_t hx[TB], hy[TB];
  anym = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    bool any = __any_sync(kFull, (alive >> (4 * t)) & 15u) != 0;
    hx[t] = __shfl_sync(kFull, Hd.x, c * TB + t);
    hy[t] = __shfl_sync(kFull, codec == C_DELTA ? Hd.z : Hd.y, c * TB + t);
    const uint32_t bw = hy[t] & 0xffu;
    if (any && bw > 32) {
      if (lane == 0) atomicOr(status, S_CORRUPT);
      any = false;
    }
    anym |= uint32_t(any) << t;
    const bool ld = any && uint32_t(lane) < bw;
    const uint32_t* src = pay + (hy[t] >> 8) + lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) v[t][k] = ld ? ld_u32<kHost>(src + uint32_t(k) * bw) : 0u;
  }
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    const uint32_t bw = hy[t] & 0xffu;
    if (codec == C_DELTA) {
      MbHdr h;
      h.first = int32_t(hx[t]);
      h.base = int32_t(__shfl_sync(kFull, Hd.y, c * TB + t));
      h.bw = bw;
      h.woff = 0;
      uint32_t w[4] = {v[t][0], v[t][1], v[t][2], v[t][3]};
      decode_mb(w, h, C_DELTA, lane, v[t]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[t][k] = unpack_lane(v[t][k], bw, lane) + hx[t];
    }
  }
}

// PREFIX step over a STR column: lengths are decoded, their exclusive scan
// gives each string's start, and the first plen bytes are compared.
template <bool kHost>
__device__ __forceinline__ void tile_prefix(const DevQuery& Q, const DevStep& S, const PageState& P,
                                            const TileHdr& Hd, TileState& T, int lane, unsigned int* status) {
  uint32_t len[TB][4];
  uint32_t anym;
  tile_decode<kHost>(Q, S.col, P, Hd, T.alive, lane, len, anym, status);
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, S.col));
  const uint8_t* bytes = pg + __shfl_sync(kFull, P.extra, S.col);
  const uint32_t plen = S.plen;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t st[4];
    excl_scan128(len[t], lane, st);
    const uint8_t* mb = bytes + __shfl_sync(kFull, Hd.sstart, S.col * TB + t);
    uint32_t match = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (((T.alive >> (4 * t + k)) & 1u) && len[t][k] >= plen) match |= 1u << k;
    for (uint32_t i = 0; i < plen; ++i) {
      if (!__any_sync(kFull, match)) break;
      const uint8_t want = S.pfx[i];
      uint8_t b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) b[k] = ((match >> k) & 1u) ? ld_u8<kHost>(mb + st[k] + i) : want;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (b[k] != want) match &= ~(1u << k);
    }
    T.alive &= ~((~match & 15u) << (4 * t));
  }
}

// Join probe step: live rows that miss are dropped; hits add this join's
// group-id contribution.
template <bool kHost>
__device__ __forceinline__ void tile_probe(const DevQuery& Q, const DevStep& S, const PageState& P,
                                           const TileHdr& Hd, TileState& T, const uint8_t* stab, int lane,
                                           unsigned int* status) {
  uint32_t v[TB][4];
  uint32_t anym;
  tile_decode<kHost>(Q, S.col, P, Hd, T.alive, lane, v, anym, status);
  if (S.ht_kind == HT_DIRECT) {
    const uint32_t width = S.smem_width;
    const uint8_t* sm = stab + S.smem_off;
    const uint32_t* gt = static_cast<const uint32_t*>(S.ht);
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      if (!((anym >> t) & 1u)) continue;
      uint32_t keep = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t off = v[t][k] - uint32_t(S.kmin);
        const bool look = ((T.alive >> (4 * t + k)) & 1u) && off < S.krange;
        uint32_t contrib = 0;
        bool hit = false;
        if (width == 1) {
          const uint32_t e = look ? uint32_t(sm[off]) : 0xffu;
          hit = e != 0xffu;
          contrib = e;
        } else if (width == 2) {
          const uint32_t e = look ? uint32_t(reinterpret_cast<const uint16_t*>(sm)[off]) : 0xffffu;
          hit = e != 0xffffu;
          contrib = e;
        } else if (width == 4) {
          const uint32_t e = look ? reinterpret_cast<const uint32_t*>(sm)[off] : kAbsent;
          hit = e != kAbsent;
          contrib = e;
        } else {
          const uint32_t e = look ? __ldg(gt + off) : kAbsent;
          hit = e != kAbsent;
          contrib = (e & 0xffffu) * S.mul0 + (e >> 16) * S.mul1;
        }
        T.gid[t][k] += hit ? contrib : 0u;
        keep |= uint32_t(hit) << k;
      }
      T.alive &= ~((~keep & 15u) << (4 * t));
    }
    return;
  }
  // open addressing: the four probes of a lane advance together
  const bool in_smem = S.smem_width != 0;
  const uint2* tab = in_smem ? reinterpret_cast<const uint2*>(stab + S.smem_off) : static_cast<const uint2*>(S.ht);
  const uint32_t mask = S.ht_mask;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t h[4], pend = 0, hit = 0, pay[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = fmix32(v[t][k]) & mask;
      pay[k] = 0;
      // the empty-slot sentinel is never a stored key
      if (((T.alive >> (4 * t + k)) & 1u) && int32_t(v[t][k]) != kEmptyKey) pend |= 1u << k;
    }
    for (uint32_t n = 0; pend && n <= mask; ++n) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((pend >> k) & 1u)) continue;
        const uint2 s = in_smem ? tab[h[k]] : __ldg(tab + h[k]);
        if (s.x == v[t][k]) {
          hit |= 1u << k;
          pay[k] = s.y;
          pend &= ~(1u << k);
        } else if (int32_t(s.x) == kEmptyKey) {
          pend &= ~(1u << k);
        } else {
          h[k] = (h[k] + 1) & mask;
        }
      }
    }
    if (pend) atomicOr(status, S_INTERNAL);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.gid[t][k] += (pay[k] & 0xffffu) * S.mul0 + (pay[k] >> 16) * S.mul1;
    const uint32_t live = (T.alive >> (4 * t)) & 15u;
    T.alive &= ~((live & ~hit & 15u) << (4 * t));
  }
}

// Predicate (RANGE / NOTRANGE / IN / FALSE) or group-key step.
template <bool kHost>
__device__ __forceinline__ void tile_filter_or_key(const DevQuery& Q, const DevStep& S, const PageState& P,
                                                   const TileHdr& Hd, TileState& T, int lane,
                                                   unsigned int* status) {
  uint32_t v[TB][4];
  uint32_t anym;
  tile_decode<kHost>(Q, S.col, P, Hd, T.alive, lane, v, anym, status);
  if (S.kind == ST_KEY) {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) T.gid[t][k] += v[t][k] * S.key_mul;
    return;
  }
  uint32_t keep = 0;
  if (S.kind == ST_RANGE || S.kind == ST_NOTRANGE) {
    const bool neg = S.kind == ST_NOTRANGE;
    // lo <= x <= hi  <=>  (x - lo) <= (hi - lo) as unsigned
    const uint32_t lo = uint32_t(S.lo), span = uint32_t(S.hi) - uint32_t(S.lo);
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) keep |= uint32_t(((v[t][k] - lo) <= span) != neg) << (4 * t + k);
  } else if (S.kind == ST_IN) {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bool hit = false;
        for (int i = 0; i < S.nin; ++i) hit |= (int32_t(v[t][k]) == S.in[i]);
        keep |= uint32_t(hit) << (4 * t + k);
      }
  }
  T.alive &= keep;
}

// ---------------------------------------------------------------------------
// Survivor lists.  After the first step the live rows of a tile are compacted
// (ballot + popc rank, the warp's selection vector) into a per-warp list in
// shared memory, entry = row-in-tile | group id << kRowBits, and every later
// step, and the aggregation, runs over the list with one survivor per lane,
// so the warp's issue slots follow the surviving rows instead of all rows.
// ---------------------------------------------------------------------------
constexpr uint32_t kTileRows = kMB * TB;
constexpr uint32_t kRowBits = 9;
static_assert(kTileRows <= (1u << kRowBits), "row index field too narrow");

// Dense first step of a tile (or none): live bits and group-id contributions.
template <bool kHost>
__device__ __forceinline__ void tile_first_step(const DevQuery& Q, const PageState& P, const TileHdr& Hd,
                                                TileState& T, const uint8_t* stab, int lane, unsigned int* status) {
  if (Q.nsteps == 0) return;
  const DevStep& S = Q.steps[0];
  if (S.kind == ST_PREFIX) tile_prefix<kHost>(Q, S, P, Hd, T, lane, status);
  else if (S.kind == ST_PROBE) tile_probe<kHost>(Q, S, P, Hd, T, stab, lane, status);
  else tile_filter_or_key<kHost>(Q, S, P, Hd, T, lane, status);
}

// Appends the tile's live rows to the warp's list; returns the list length.
__device__ __forceinline__ uint32_t tile_compact(const TileState& T, uint32_t* list, int lane) {
  uint32_t n = 0;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool live = (T.alive >> (4 * t + k)) & 1u;
      const uint32_t m = __ballot_sync(kFull, live);
      if (live) list[n + __popc(m & lt)] = uint32_t(t * kMB + k * 32 + lane) | (T.gid[t][k] << kRowBits);
      n += __popc(m);
    }
  __syncwarp();
  return n;
}

// Value of FOR/DICT column c at tile row r: one bit-field read from the
// packed payload (two words when the field straddles them).
template <bool kHost>
__device__ __forceinline__ uint32_t point_value(const DevQuery& Q, int c, const PageState& P, const TileHdr& Hd,
                                                uint32_t r, bool valid) {
  const uint32_t codec = Q.cols[c].codec;
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(codec, P.prow));
  const int src = c * TB + int(r >> 7);
  const uint32_t base = __shfl_sync(kFull, Hd.x, src);
  const uint32_t wob = __shfl_sync(kFull, Hd.y, src);
  const uint32_t bw = tmin<uint32_t>(wob & 0xffu, 32u);
  uint32_t x = 0;
  if (valid && bw != 0) {
    const uint32_t bit = (r & (kMB - 1)) * bw;
    const uint32_t* p = pay + (wob >> 8) + (bit >> 5);
    const uint32_t sh = bit & 31u;
    const uint32_t lo = ld_u32<kHost>(p);
    const uint32_t hi = sh + bw > 32 ? ld_u32<kHost>(p + 1) : 0u;
    x = __funnelshift_r(lo, hi, sh);
    if (bw < 32) x &= (1u << bw) - 1u;
  }
  return base + x;
}

// Value of any integer column at tile row r.  DELTA columns need the prefix
// sum of their mini block, so the mini blocks holding the round's rows are
// decoded densely and each lane picks its row with shuffles.
template <bool kHost>
__device__ __forceinline__ uint32_t row_value(const DevQuery& Q, int c, const PageState& P, const TileHdr& Hd,
                                              uint32_t r, bool valid, int lane, unsigned int* status) {
  if (Q.cols[c].codec != C_DELTA) return point_value<kHost>(Q, c, P, Hd, r, valid);
  const uint32_t need = __reduce_or_sync(kFull, valid ? 1u << (r >> 7) : 0u);
  uint32_t alive = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
    if ((need >> t) & 1u) alive |= 15u << (4 * t);
  uint32_t v[TB][4], anym;
  tile_decode<kHost>(Q, c, P, Hd, alive, lane, v, anym, status);
  uint32_t out = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = __shfl_sync(kFull, v[t][k], int(r & 31));
      if ((r >> 5) == uint32_t(t * 4 + k)) out = x;
    }
  }
  return out;
}

// PREFIX on a list: lengths and starts of the round's mini blocks are
// decoded densely and gathered per lane, then the bytes are compared.
template <bool kHost>
__device__ __forceinline__ bool row_prefix(const DevQuery& Q, const DevStep& S, const PageState& P,
                                           const TileHdr& Hd, uint32_t r, bool valid, int lane,
                                           unsigned int* status) {
  const uint32_t need = __reduce_or_sync(kFull, valid ? 1u << (r >> 7) : 0u);
  uint32_t alive = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
    if ((need >> t) & 1u) alive |= 15u << (4 * t);
  uint32_t len[TB][4], anym;
  tile_decode<kHost>(Q, S.col, P, Hd, alive, lane, len, anym, status);
  uint32_t my_len = 0, my_start = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t st[4];
    excl_scan128(len[t], lane, st);
    const uint32_t mb_start = __shfl_sync(kFull, Hd.sstart, S.col * TB + t);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t l = __shfl_sync(kFull, len[t][k], int(r & 31));
      const uint32_t s0 = __shfl_sync(kFull, st[k], int(r & 31));
      if ((r >> 5) == uint32_t(t * 4 + k)) {
        my_len = l;
        my_start = mb_start + s0;
      }
    }
  }
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, S.col));
  const uint8_t* bytes = pg + __shfl_sync(kFull, P.extra, S.col) + my_start;
  bool match = valid && my_len >= S.plen;
  for (uint32_t i = 0; i < S.plen; ++i) {
    if (!__any_sync(kFull, match)) break;
    if (match && ld_u8<kHost>(bytes + i) != S.pfx[i]) match = false;
  }
  return match;
}

// Join probe of one key; on a hit adds the join's group-id contribution.
__device__ __forceinline__ bool row_probe(const DevStep& S, const uint8_t* stab, uint32_t key, bool valid,
                                          uint32_t& gid, unsigned int* status) {
  if (!valid) return false;
  if (S.ht_kind == HT_DIRECT) {
    const uint32_t off = key - uint32_t(S.kmin);
    if (off >= S.krange) return false;
    uint32_t e;
    switch (S.smem_width) {
      case 1: e = stab[S.smem_off + off]; if (e == 0xffu) return false; gid += e; return true;
      case 2: e = reinterpret_cast<const uint16_t*>(stab + S.smem_off)[off]; if (e == 0xffffu) return false; gid += e; return true;
      case 4: e = reinterpret_cast<const uint32_t*>(stab + S.smem_off)[off]; if (e == kAbsent) return false; gid += e; return true;
      default:
        e = __ldg(static_cast<const uint32_t*>(S.ht) + off);
        if (e == kAbsent) return false;
        gid += (e & 0xffffu) * S.mul0 + (e >> 16) * S.mul1;
        return true;
    }
  }
  if (int32_t(key) == kEmptyKey) return false;
  const uint2* tab = S.smem_width ? reinterpret_cast<const uint2*>(stab + S.smem_off) : static_cast<const uint2*>(S.ht);
  uint32_t pay;
  if (!ht_probe(tab, S.ht_mask, int32_t(key), &pay, status)) return false;
  gid += (pay & 0xffffu) * S.mul0 + (pay >> 16) * S.mul1;
  return true;
}

// Steps 1.. of the query over the warp's list; returns the list length.
template <bool kHost>
__device__ __forceinline__ uint32_t list_steps(const DevQuery& Q, const PageState& P, const TileHdr& Hd,
                                               uint32_t* list, uint32_t n, const uint8_t* stab, int lane,
                                               unsigned int* status) {
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t s = 1; s < Q.nsteps && n != 0; ++s) {
    const DevStep& S = Q.steps[s];
    uint32_t out = 0;
    for (uint32_t i0 = 0; i0 < n; i0 += 32) {
      const bool valid = i0 + lane < n;
      const uint32_t e = valid ? list[i0 + lane] : 0u;
      const uint32_t r = e & ((1u << kRowBits) - 1u);
      uint32_t gid = e >> kRowBits;
      bool keep;
      if (S.kind == ST_PREFIX) {
        keep = row_prefix<kHost>(Q, S, P, Hd, r, valid, lane, status);
      } else {
        const uint32_t v = row_value<kHost>(Q, S.col, P, Hd, r, valid, lane, status);
        if (S.kind == ST_PROBE) {
          keep = row_probe(S, stab, v, valid, gid, status);
        } else if (S.kind == ST_KEY) {
          gid += v * S.key_mul;
          keep = valid;
        } else {
          keep = valid && step_pred(S, int32_t(v));
        }
      }
      const uint32_t m = __ballot_sync(kFull, keep);
      __syncwarp();
      if (keep) list[out + __popc(m & lt)] = r | (gid << kRowBits);
      out += __popc(m);
    }
    __syncwarp();
    n = out;
  }
  return n;
}

}  // namespace dpf

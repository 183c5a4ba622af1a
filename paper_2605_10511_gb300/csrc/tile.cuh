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
    if (is_str_codec(C.codec)) P.extra = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(P.pg + 12));
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
      if (is_str_codec(codec))
        h.sstart = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(
            pg + kPageHdr + uint64_t(P.nmb_page) * 8 + uint64_t(i0 + ht) * 4));
    }
  }
  return h;
}

// ------------------------------------------------------------------ staging
// The IO stage of Sec. 3.2 overlapped with decompression: the first step's
// compressed mini blocks are copied HBM -> shared memory with cp.async (16
// bytes per lane, through L2 only) into a per-warp ring, one tile ahead of
// the decode for the packed words and two tiles ahead for the mini block
// headers (a tile's word copies need its headers' offsets and widths).  A
// warp waits only for its own copies (cp.async.wait_group, no spinning) and
// decodes from shared memory, so the loads of the next tile are in flight
// while this one is decoded, probed and compacted, and hold no registers.
// Ring of one warp, for slots of up to bwcap bits a value: 3 header slots of
// TB headers (16 bytes each at most), then 2 word slots of TB mini blocks of
// 4 * (bwcap + 1) words (a mini block's 4 * bw words plus one spare group).
constexpr uint32_t kStageHdrSlot = TB * 16;
__host__ __device__ constexpr uint32_t stage_pw(uint32_t bwcap) { return 4u * (bwcap + 1u); }
__host__ __device__ constexpr uint32_t stage_warp_bytes(uint32_t bwcap) {
  return bwcap == 0 ? 0u : 3u * kStageHdrSlot + 2u * TB * 4u * stage_pw(bwcap);
}
__device__ __forceinline__ uint8_t* stage_hdr(uint8_t* ring, uint32_t slot) { return ring + slot * kStageHdrSlot; }
__device__ __forceinline__ uint32_t* stage_words(uint8_t* ring, uint32_t slot, uint32_t bwcap) {
  return reinterpret_cast<uint32_t*>(ring + 3 * kStageHdrSlot) + slot * TB * stage_pw(bwcap);
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }

// Byte offset of mini block i0's header inside its header slot: the copy
// starts at the 16-byte boundary at or below the header (8-byte headers of
// an odd mini block start 8 bytes into a chunk).
__device__ __forceinline__ uint32_t stage_hdr_skew(uint32_t codec, uint32_t i0) {
  return (kPageHdr + i0 * mb_hdr_bytes(codec)) & 15u;
}

// Copies the headers of mini blocks [i0, i0 + nmb) of a page of column
// codec (at pg) into header slot `slot`: the 16-byte chunks that cover them,
// from the boundary at or below the first (pages are 16-aligned) to at most
// the 16-aligned end of the header array (the payload follows it), so every
// chunk lies inside the page.
__device__ __forceinline__ void stage_headers(uint8_t* ring, uint32_t slot, const uint8_t* pg, uint32_t codec,
                                              uint32_t i0, uint32_t nmb, int lane) {
  const uint32_t hb = mb_hdr_bytes(codec);
  const uint64_t first = kPageHdr + uint64_t(i0) * hb;
  const uint32_t skew = uint32_t(first & 15u);
  const uint32_t chunks = (skew + nmb * hb + 15) / 16;  // <= 3 (8-byte) or 4 (16-byte headers)
  if (uint32_t(lane) < chunks)
    cp_async16(stage_hdr(ring, slot) + lane * 16, pg + (first - skew) + uint32_t(lane) * 16);
}

// Copies the packed words of the nmb mini blocks whose headers sit in header
// slot hslot into word slot wslot: a mini block of bit width bw is 4 * bw
// words = bw 16-byte chunks (16-aligned: load validation checks the word
// offsets), lane i copying chunk i.  Mini blocks wider than the ring's slots
// are left out (the decode reports them).
__device__ __forceinline__ void stage_payload(uint8_t* ring, uint32_t bwcap, uint32_t hslot, uint32_t wslot,
                                              const uint8_t* pay, uint32_t codec, uint32_t i0, uint32_t nmb,
                                              int lane) {
  const uint8_t* hs = stage_hdr(ring, hslot) + stage_hdr_skew(codec, i0);
  uint32_t* dst = stage_words(ring, wslot, bwcap);
  const uint32_t pw = stage_pw(bwcap);
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (t >= int(nmb)) break;
    const uint32_t wob = codec == C_DELTA ? reinterpret_cast<const uint32_t*>(hs + t * 16)[2]
                                          : reinterpret_cast<const uint32_t*>(hs + t * 8)[1];
    const uint32_t bw = wob & 0xffu;
    if (uint32_t(lane) < bw && bw <= bwcap)
      cp_async16(dst + t * pw + uint32_t(lane) * 4, pay + uint64_t(wob >> 8) * 4 + uint32_t(lane) * 16);
  }
}

// The tile's headers of column c from header slot hslot, laid out as
// load_headers lays them (lane c * TB + t holds mini block t's header).
__device__ __forceinline__ TileHdr staged_headers(uint8_t* ring, uint32_t hslot, int c, uint32_t codec, uint32_t i0,
                                                  uint32_t nmb, int lane) {
  TileHdr h{0, 0, 0, 0};
  const int ht = lane % TB;
  if (lane / TB == c && ht < int(nmb)) {
    const uint8_t* hs = stage_hdr(ring, hslot) + stage_hdr_skew(codec, i0);
    if (codec == C_DELTA) {
      const uint4 v = *reinterpret_cast<const uint4*>(hs + ht * 16);
      h.x = v.x;
      h.y = v.y;
      h.z = v.z;
    } else {
      const uint2 v = *reinterpret_cast<const uint2*>(hs + ht * 8);
      h.x = v.x;
      h.y = v.y;
    }
  }
  return h;
}

// L2 prefetch of the headers of mini blocks [i0, i0 + nmb) of every column
// but c (the later steps read them per survivor).
__device__ __forceinline__ void prefetch_other_headers(const DevQuery& Q, const PageState& P, int c, uint32_t i0,
                                                       uint32_t nmb, int lane) {
  const int hc = lane / TB, ht = lane % TB;
  const uint64_t hpg = __shfl_sync(kFull, P.pg, hc < int(Q.ncols) ? hc : 0);
  if (hc < int(Q.ncols) && hc != c && ht < int(nmb))
    prefetch_l2(reinterpret_cast<const uint8_t*>(hpg) + kPageHdr + uint64_t(i0 + ht) * mb_hdr_bytes(Q.cols[hc].codec));
}

// The staged words of the tile being decoded: mini block t's words at
// p + t * pw (in page order), slots of up to bwcap bits.
struct StagedPay {
  const uint32_t* p;
  uint32_t pw, bwcap;
};

// L2 prefetch of the packed words of mini blocks [i0, i0 + nmb) of column
// c (its headers in Hd, lanes c * TB + t): every 128-byte line of each block.
__device__ __forceinline__ void prefetch_words(const DevQuery& Q, const PageState& P, const TileHdr& Hd, int c,
                                               uint32_t nmb, int lane) {
  const int t = lane % TB, part = lane / TB;  // up to 8 lanes per block: lines part, part + 8, ...
  const uint32_t codec = Q.cols[c].codec;
  const uint32_t wob = __shfl_sync(kFull, codec == C_DELTA ? Hd.z : Hd.y, c * TB + t);
  const uint64_t pg = __shfl_sync(kFull, P.pg, c);
  if (t >= int(nmb) || codec == C_FOR64 || is_str_codec(codec)) return;
  const uint32_t bw = tmin<uint32_t>(wob & 0xffu, 32u), bytes = 16 * bw;
  const uint8_t* w = reinterpret_cast<const uint8_t*>(pg) + payload_offset(codec, P.prow) + uint64_t(wob >> 8) * 4;
  for (uint32_t off = uint32_t(part) * 128; off < bytes; off += (32 / TB) * 128) prefetch_l2(w + off);
}

struct TileState {
  uint32_t alive;         // bit 4t+k: row 32k+lane of mini block t is live
  uint32_t gid[TB][4];    // dense group id of each row
};

// kGid = false: the tile's dense step adds no group-id contribution, so the
// group ids stay 0 and are neither kept nor written to the list.
template <bool kGid = true>
__device__ __forceinline__ void tile_init(const PageState& P, uint32_t i0, uint32_t nmb, int lane,
                                          TileState& T) {
  if (kGid) {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) T.gid[t][k] = 0;
  }
  if (nmb == uint32_t(TB) && (i0 + TB) * kMB <= P.prow) {  // a full tile
    T.alive = (TB == 8) ? 0xffffffffu : ((1u << (4 * TB)) - 1u);
    return;
  }
  T.alive = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t r = (i0 + t) * kMB + k * 32 + lane;
      if (t < int(nmb) && r < P.prow) T.alive |= 1u << (4 * t + k);
    }
}

// Loads and decodes column c for the mini blocks with live rows: v[t][k]
// = value of row 32k + lane of mini block t (the payload words are loaded
// into v and decoded in place).  anym bit t = mini block t was decoded.
// Specialised on the codec (FOR/DICT/STR lengths vs DELTA) so the unrolled
// loops carry no per-value branch on it.
template <bool kHost, bool kDelta, bool kStaged = false>
__device__ __forceinline__ void decode_t(const DevQuery& Q, int c, const PageState& P, const TileHdr& Hd,
                                         uint32_t alive, int lane, uint32_t (&v)[TB][4], uint32_t& anym,
                                         unsigned int* status, StagedPay sp = StagedPay{nullptr, 0, 0}) {
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(Q.cols[c].codec, P.prow));
  uint32_t hx[TB], hy[TB];
  anym = 0;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    bool any = __any_sync(kFull, (alive >> (4 * t)) & 15u) != 0;
    hx[t] = __shfl_sync(kFull, Hd.x, c * TB + t);
    hy[t] = __shfl_sync(kFull, kDelta ? Hd.z : Hd.y, c * TB + t);
    const uint32_t bw = hy[t] & 0xffu;
    if (any && bw > 32) {
      if (lane == 0) atomicOr(status, S_CORRUPT);
      any = false;
    }
    if (kStaged && any && bw > sp.bwcap) {  // the ring is sized from the column's widest mini block
      if (lane == 0) atomicOr(status, S_INTERNAL);
      any = false;
    }
    anym |= uint32_t(any) << t;
    const bool ld = any && uint32_t(lane) < bw;
    if (kStaged) {
      const uint32_t* src = sp.p + t * sp.pw + lane;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[t][k] = ld ? src[uint32_t(k) * bw] : 0u;
    } else {
      const uint32_t* src = pay + (hy[t] >> 8) + lane;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[t][k] = ld ? ld_u32<kHost>(src + uint32_t(k) * bw) : 0u;
    }
  }
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    const uint32_t bw = hy[t] & 0xffu;
#pragma unroll
    for (int k = 0; k < 4; ++k) v[t][k] = unpack_lane(v[t][k], bw, lane);
    if (kDelta) {
      // x_j = first + sum_{i<=j} (dmin + p_i), modulo 2^32
      const uint32_t dmin = __shfl_sync(kFull, Hd.y, c * TB + t);
      uint32_t carry = hx[t];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t s = warp_incl_scan(v[t][k] + dmin, lane);
        v[t][k] = carry + s;
        carry += __shfl_sync(kFull, s, 31);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[t][k] += hx[t];
    }
  }
}

template <bool kHost>
__device__ __forceinline__ void tile_decode(const DevQuery& Q, int c, const PageState& P, const TileHdr& Hd,
                                            uint32_t alive, int lane, uint32_t (&v)[TB][4], uint32_t& anym,
                                            unsigned int* status) {
  if (Q.cols[c].codec == C_DELTA) decode_t<kHost, true>(Q, c, P, Hd, alive, lane, v, anym, status);
  else decode_t<kHost, false>(Q, c, P, Hd, alive, lane, v, anym, status);
}

// ------------------------------------------------------------ strings
// A string predicate on one stored string: PREFIX compares its first plen
// bytes; CONTAINS runs the Knuth-Morris-Pratt automaton of the pattern over
// all its bytes (the matcher Sec. 4.1 integrates for LIKE).  FSST strings
// are decoded on the fly, symbol by symbol (code < nsym: the symbol's bytes;
// code 255: the next stored byte), and never written anywhere.
// Scan kinds of string_scan: ST_PREFIX, ST_CONTAINS (KMP), and a CONTAINS
// of at most 8 bytes compared through a sliding window.
constexpr int kScanContainsShort = 256;

struct StrMatch {
  const DevStep* S;
  uint32_t pos = 0;     // PREFIX: bytes matched; CONTAINS (KMP): automaton state
  uint64_t win = 0;     // CONTAINS of <= 8 bytes: the last 8 bytes seen
  bool hit = false;
  // Feeds one decoded byte; returns false once the outcome is decided.
  template <int kKind>
  __device__ __forceinline__ bool feed(uint8_t b) {
    if (kKind == ST_PREFIX) {
      if (b != S->pfx[pos]) return false;
      if (++pos == S->plen) { hit = true; return false; }
      return true;
    }
    if (kKind == kScanContainsShort) {  // short pattern: compare a sliding window
      win = (win << 8) | b;
      ++pos;
      const uint64_t pat = uint32_t(S->in[0]) | (uint64_t(uint32_t(S->in[1])) << 32);
      const uint64_t mask = S->plen >= 8 ? ~0ull : ((1ull << (8 * S->plen)) - 1);
      if (pos >= S->plen && (win & mask) == pat) { hit = true; return false; }
      return true;
    }
    uint32_t q = pos;
    while (q > 0 && b != S->pfx[q]) q = S->kmp[q - 1];
    if (b == S->pfx[q]) ++q;
    pos = q;
    if (q == S->plen) { hit = true; return false; }
    return true;
  }
};

template <bool kHost, int kKind>
__device__ __forceinline__ bool string_scan(const DevStep& S, const uint8_t* s, uint32_t len, const int4* sym) {
  StrMatch m;
  m.S = &S;
  if (sym == nullptr) {                                 // STR: raw bytes
    // 4-byte aligned words cover the string (inside the 16-byte padded page)
    const uint8_t* w0 = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(s) & ~uintptr_t(3));
    const uint8_t* end = s + len;
    uint32_t skip = uint32_t(s - w0);
    for (const uint8_t* w = w0; w < end; w += 4) {
      uint32_t x = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(w)) >> (8 * skip);
      const uint32_t nb = tmin<uint32_t>(4u - skip, uint32_t(end - (w + skip)));
      skip = 0;
      bool go = true;
      for (uint32_t k = 0; k < nb && go; ++k, x >>= 8) go = m.template feed<kKind>(uint8_t(x));
      if (!go) break;
    }
    return m.hit;
  }
  for (uint32_t i = 0; i < len;) {                      // FSST: decode symbol by symbol
    const uint32_t c = ld_u8<kHost>(s + i++);
    if (c == kFsstEscape) {                             // load-time validation: a literal follows
      if (!m.template feed<kKind>(ld_u8<kHost>(s + i++))) break;
      continue;
    }
    const int4 e = __ldg(sym + c);                      // load-time validation: c < nsym
    uint64_t w = uint32_t(e.x) | (uint64_t(uint32_t(e.y)) << 32);
    bool go = true;
    for (int k = 0; k < e.z && go; ++k, w >>= 8) go = m.template feed<kKind>(uint8_t(w));
    if (!go) break;
  }
  return m.hit;
}

// Code-level matching of an FSST string (LIKE on compressed strings): the
// matcher's state advances by one table lookup per code instead of per
// decoded byte.  `tab` (shared memory, built by build_fsst_matcher) holds,
// for every state q < plen, the entry after symbol code c at tab[q * 256 + c]
// and after escaped literal byte b at tab[(plen + 1) * 256 + q * 256 + b];
// an entry is the next state, kFsstHit (the pattern was completed inside the
// symbol) or kFsstDead (a PREFIX mismatch).  The string's bytes are read as
// aligned 4-byte words (inside the 16-byte padded page).
constexpr uint8_t kFsstHit = 0x80, kFsstDead = 0x7f;
template <bool kHost>
__device__ __forceinline__ bool fsst_table_match(const DevStep& S, const uint8_t* s, uint32_t len, const uint8_t* tab) {
  const uint8_t* btab = tab + (uint32_t(S.plen) + 1) * 256;
  const uint8_t* w0 = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(s) & ~uintptr_t(3));
  const uint8_t* end = s + len;
  uint32_t skip = uint32_t(s - w0), q = 0;
  bool esc = false;
  for (const uint8_t* w = w0; w < end; w += 4) {
    uint32_t x = ld_u32<kHost>(reinterpret_cast<const uint32_t*>(w)) >> (8 * skip);
    const uint32_t nb = tmin<uint32_t>(4u - skip, uint32_t(end - (w + skip)));
    skip = 0;
    for (uint32_t k = 0; k < nb; ++k, x >>= 8) {
      const uint32_t c = x & 0xffu;
      uint32_t e;
      if (esc) {
        e = btab[q * 256 + c];
        esc = false;
      } else if (c == kFsstEscape) {
        esc = true;
        continue;
      } else {
        e = tab[q * 256 + c];
      }
      if (e & kFsstHit) return true;
      if (e == kFsstDead) return false;
      q = e;
    }
  }
  return false;
}

// The matcher state after feeding byte b in state q < plen: the next state,
// kFsstHit when the pattern completes, kFsstDead when a PREFIX cannot match.
__device__ __forceinline__ uint32_t matcher_feed(const DevStep& S, uint32_t q, uint32_t b) {
  if (S.kind == ST_PREFIX) {
    if (b != S.pfx[q]) return kFsstDead;
  } else {  // CONTAINS: the Knuth-Morris-Pratt automaton
    while (q > 0 && b != S.pfx[q]) q = S.kmp[q - 1];
    if (b != S.pfx[q]) return q;
  }
  return q + 1 == S.plen ? uint32_t(kFsstHit) : q + 1;
}

// Builds step S's code-level tables at tab (all threads of the CTA): for
// every state q < plen, each of the column's nsym symbols fed byte by byte
// (codes >= nsym never occur: load validation), and each literal byte.
__device__ __forceinline__ void build_fsst_matcher(const DevStep& S, const int4* sym, uint32_t nsym, uint8_t* tab) {
  const uint32_t plen = S.plen, n = plen * 256;
  uint8_t* btab = tab + (plen + 1) * 256;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t q = i >> 8, c = i & 255u;
    btab[i] = uint8_t(matcher_feed(S, q, c));
    uint32_t e = kFsstDead;
    if (c < nsym) {
      const int4 y = __ldg(sym + c);
      uint64_t w = uint32_t(y.x) | (uint64_t(uint32_t(y.y)) << 32);
      e = q;
      for (int k = 0; k < y.z; ++k, w >>= 8) {
        e = matcher_feed(S, e, uint32_t(w & 0xffu));
        if (e == kFsstHit || e == kFsstDead) break;
      }
    }
    tab[i] = uint8_t(e);
  }
}

// SQL LIKE of a raw string s[0..n) against pfx[0..plen): '%' any run of
// bytes, '_' any one byte.  The iterative greedy wildcard matcher: literals
// and '_' advance both sides; a '%' records where it stands and first
// matches nothing; on a mismatch the last '%' takes one more byte and the
// match resumes after it.  O(n * plen) at worst, no recursion.
template <bool kHost>
__device__ __forceinline__ bool like_match(const DevStep& S, const uint8_t* s, uint32_t n) {
  const uint32_t m = S.plen, none = 0xffffffffu;
  uint32_t i = 0, j = 0, star_j = none, star_i = 0;
  while (i < n) {
    const uint32_t pc = j < m ? S.pfx[j] : 0u;
    if (j < m && pc != '%' && (pc == '_' || pc == ld_u8<kHost>(s + i))) {
      ++i;
      ++j;
    } else if (j < m && pc == '%') {
      star_j = j++;
      star_i = i;
    } else if (star_j != none) {
      j = star_j + 1;
      i = ++star_i;
    } else {
      return false;
    }
  }
  while (j < m && S.pfx[j] == '%') ++j;
  return j == m;
}

template <bool kHost>
__device__ __forceinline__ bool string_match(const DevStep& S, const uint8_t* s, uint32_t len, const int4* sym,
                                             const uint8_t* tab = nullptr) {
  if (S.kind == ST_LIKE) return sym == nullptr && like_match<kHost>(S, s, len);  // STR columns only
  if (S.plen == 0) return true;                         // an empty pattern matches
  if (tab != nullptr) return fsst_table_match<kHost>(S, s, len, tab);
  if (S.kind == ST_PREFIX) {
    if (sym == nullptr && len < S.plen) return false;
    return string_scan<kHost, ST_PREFIX>(S, s, len, sym);
  }
  if (S.plen <= 8) return string_scan<kHost, kScanContainsShort>(S, s, len, sym);
  return string_scan<kHost, ST_CONTAINS>(S, s, len, sym);
}

// PREFIX / CONTAINS step over a string column, dense: lengths decoded, their
// exclusive scan gives each string's start, then each live row's string is
// matched.  kText = false compiles the raw-PREFIX path only (the general
// matcher of CONTAINS and FSST is left out of the kernel's code); the host
// launches that build only for batches without such steps, and a step it
// cannot run drops its rows and reports S_INTERNAL.
template <bool kHost, bool kText = true>
__device__ __forceinline__ void tile_prefix(const DevQuery& Q, const DevStep& S, const PageState& P,
                                            const TileHdr& Hd, TileState& T, int lane, unsigned int* status,
                                            const uint8_t* stab) {
  uint32_t len[TB][4];
  uint32_t anym;
  tile_decode<kHost>(Q, S.col, P, Hd, T.alive, lane, len, anym, status);
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, S.col));
  const uint8_t* bytes = pg + __shfl_sync(kFull, P.extra, S.col);
  const int4* sym = Q.cols[S.col].codec == C_FSST ? Q.cols[S.col].sym : nullptr;
  const uint8_t* tab = sym != nullptr && S.smem_width ? stab + S.smem_off : nullptr;
  const bool lockstep = S.kind == ST_PREFIX && sym == nullptr;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t st[4];
    excl_scan128(len[t], lane, st);
    const uint8_t* mb = bytes + __shfl_sync(kFull, Hd.sstart, S.col * TB + t);
    uint32_t match = 0;
    if (lockstep) {
      // raw PREFIX: the warp compares byte i of all its rows' strings at once
      const uint32_t plen = S.plen;
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
    } else {
      if constexpr (kText) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (((T.alive >> (4 * t + k)) & 1u) && string_match<kHost>(S, mb + st[k], len[t][k], sym, tab))
            match |= 1u << k;
      } else {
        if (lane == 0) atomicOr(status, S_INTERNAL);
      }
    }
    T.alive &= ~((~match & 15u) << (4 * t));
  }
}

// Probe modes: direct table copied into shared memory as 1/2/4-byte group-id
// contributions, direct or rank-directory table in global memory, open
// addressing (shared or global slots).
enum ProbeMode : int { PM_S1 = 0, PM_S2 = 1, PM_S4 = 2, PM_GDIRECT = 3, PM_OPEN = 4 };
__device__ __forceinline__ int probe_mode(const DevStep& S) {
  if (S.ht_kind == HT_OPEN) return PM_OPEN;
  return S.smem_width == 1 ? PM_S1 : S.smem_width == 2 ? PM_S2 : S.smem_width == 4 ? PM_S4 : PM_GDIRECT;
}

// Direct-table probe of one key: true on a hit, which adds the join's
// group-id contribution to gid.
template <int kMode, bool kContrib = true>
__device__ __forceinline__ bool probe_direct(const DevStep& S, const uint8_t* stab, uint32_t key, bool valid,
                                             uint32_t& gid) {
  const uint32_t off = key - uint32_t(S.kmin);
  const bool look = valid && off < S.krange;
  uint32_t e;
  bool hit;
  if (kMode == PM_S1) {
    e = look ? uint32_t(stab[S.smem_off + off]) : 0xffu;
    hit = e != 0xffu;
  } else if (kMode == PM_S2) {
    e = look ? uint32_t(reinterpret_cast<const uint16_t*>(stab + S.smem_off)[off]) : 0xffffu;
    hit = e != 0xffffu;
  } else if (kMode == PM_S4) {
    e = look ? reinterpret_cast<const uint32_t*>(stab + S.smem_off)[off] : kAbsent;
    hit = e != kAbsent;
  } else {  // a table in device memory: direct, or a rank directory
    if (S.ht_kind == HT_RANK) e = look ? rank_entry(S.ht, S.krange, off) : kAbsent;
    else e = look ? __ldg(static_cast<const uint32_t*>(S.ht) + off) : kAbsent;
    hit = e != kAbsent;
    e = kContrib ? (e & 0xffffu) * S.mul0 + (e >> 16) * S.mul1 : 0u;
  }
  if (kContrib) gid += hit ? e : 0u;
  return hit;
}

// Dense probe of a rank-directory table: the presence-bit words of the
// tile's rows are loaded first, all independent of one another; then, only
// when the step adds group-id contributions, each hit's running count and
// its payload.  Dead and out-of-range rows read directory word 0 and count
// as misses; a miss reads no count and no payload.
template <bool kContrib>
__device__ __forceinline__ void dense_probe_rank(const DevStep& S, const uint32_t (&v)[TB][4], uint32_t anym,
                                                 TileState& T) {
  const uint32_t* dw = static_cast<const uint32_t*>(S.ht);
  const uint32_t* pay = dw + 4 * ((uint64_t(S.krange) + 63) >> 6);
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    if (!((anym >> t) & 1u)) continue;
    uint32_t keep = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t off = v[t][k] - uint32_t(S.kmin);
      const bool look = off < S.krange;
      const uint32_t wi = look ? rank_bits_word(off) : 0u;
      const uint32_t bits = __ldg(dw + wi);
      const bool hit = look && ((bits >> (off & 31u)) & 1u);
      keep |= uint32_t(hit) << k;
      if (kContrib) {
        const uint32_t idx = hit ? __ldg(dw + wi + 2) + uint32_t(__popc(bits & ((1u << (off & 31u)) - 1u))) : 0u;
        const uint32_t e = hit ? __ldg(pay + idx) : 0u;
        T.gid[t][k] += hit ? (e & 0xffffu) * S.mul0 + (e >> 16) * S.mul1 : 0u;
      }
    }
    T.alive &= ~((~keep & 15u) << (4 * t));
  }
}

// Join probe step over a decoded tile: live rows that miss are dropped;
// hits add this join's group-id contribution.
template <int kMode, bool kContrib = true>
__device__ __forceinline__ void dense_probe(const DevStep& S, const uint8_t* stab, const uint32_t (&v)[TB][4],
                                            uint32_t anym, TileState& T, unsigned int* status) {
  if (kMode != PM_OPEN) {
    // every row is probed (the bounds check keeps dead rows' lookups inside
    // the table); the result is masked with the live bits
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      if (!((anym >> t) & 1u)) continue;
      uint32_t keep = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        keep |= uint32_t(probe_direct<kMode, kContrib>(S, stab, v[t][k], true, T.gid[t][k])) << k;
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
    if (kContrib) {
#pragma unroll
      for (int k = 0; k < 4; ++k) T.gid[t][k] += (pay[k] & 0xffffu) * S.mul0 + (pay[k] >> 16) * S.mul1;
    }
    const uint32_t live = (T.alive >> (4 * t)) & 15u;
    T.alive &= ~((live & ~hit & 15u) << (4 * t));
  }
}

// Dense step over one tile, specialised on the column's codec: a probe, a
// group key or a predicate (RANGE / NOTRANGE / IN / FALSE).
// Mini blocks of column c in the tile (bit t) whose values all lie outside
// [zlo, zhi], from their headers alone: FOR/DICT values lie in
// [base, base + 2^bw - 1]; a DELTA mini block's values lie within 127 steps
// of its first value, each step in [min(0, dmin), max(0, dmin + 2^bw - 1)]
// (used only when that bound stays inside int32, i.e. nothing wrapped).
template <bool kDelta>
__device__ __forceinline__ uint32_t pruned_mbs(const TileHdr& Hd, int c, int32_t zlo, int32_t zhi, int lane) {
  bool out = false;
  if (lane / TB == c) {
    int64_t lo, hi;
    if (kDelta) {
      const int64_t first = int32_t(Hd.x), dmin = int32_t(Hd.y);
      const uint32_t bw = tmin<uint32_t>(Hd.z & 0xffu, 32u);
      const int64_t span = bw >= 32 ? int64_t(0xffffffffll) : (int64_t(1) << bw) - 1;
      lo = first + 127 * tmin<int64_t>(0, dmin);
      hi = first + 127 * tmax<int64_t>(0, dmin + span);
      if (lo < INT32_MIN || hi > INT32_MAX) {
        lo = INT32_MIN;
        hi = INT32_MAX;
      }
    } else {
      const uint32_t bw = tmin<uint32_t>(Hd.y & 0xffu, 32u);
      lo = int32_t(Hd.x);
      hi = lo + (bw >= 32 ? int64_t(0xffffffffll) : (int64_t(1) << bw) - 1);
    }
    out = zlo > zhi || hi < int64_t(zlo) || lo > int64_t(zhi);
  }
  return (__ballot_sync(kFull, out) >> (c * TB)) & ((1u << TB) - 1u);
}

// ---- staged dense step: one mini block at a time from the staging ring ----
// With the words in shared memory, a lane extracts its four values directly
// (value 32k + lane sits at bit (32k + lane) * bw of the mini block: two
// shared loads and a funnel shift, no shuffles), and each mini block is
// decoded, tested and folded into the live bits before the next, so only
// four values per lane are live instead of sixteen.

// Decodes mini block t of column c (header in Hd's lane c * TB + t) into
// v[k] = value of row 32k + lane; false when the block has no live row (or
// cannot be decoded: the status word says why).
template <bool kDelta>
__device__ __forceinline__ bool staged_mb_decode(const TileHdr& Hd, int c, int t, uint32_t alive, StagedPay sp,
                                                 int lane, uint32_t (&v)[4], unsigned int* status) {
  bool any = __any_sync(kFull, (alive >> (4 * t)) & 15u) != 0;
  const uint32_t hx = __shfl_sync(kFull, Hd.x, c * TB + t);
  const uint32_t hy = __shfl_sync(kFull, kDelta ? Hd.z : Hd.y, c * TB + t);
  const uint32_t bw = hy & 0xffu;
  if (any && (bw > 32 || bw > sp.bwcap)) {
    if (lane == 0) atomicOr(status, bw > 32 ? S_CORRUPT : S_INTERNAL);
    any = false;
  }
  if (!any) return false;
  const uint32_t* src = sp.p + t * sp.pw;
  const uint32_t bit = uint32_t(lane) * bw, w = bit >> 5, sh = bit & 31u;
  const uint32_t mask = bw >= 32 ? 0xffffffffu : (1u << bw) - 1u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t* q = src + uint32_t(k) * bw + w;  // the word after a block's last is inside the slot
    v[k] = __funnelshift_r(q[0], q[1], sh) & mask;
  }
  if (kDelta) {
    // x_j = first + sum_{i<=j} (dmin + p_i), modulo 2^32
    const uint32_t dmin = __shfl_sync(kFull, Hd.y, c * TB + t);
    uint32_t carry = hx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t sc = warp_incl_scan(v[k] + dmin, lane);
      v[k] = carry + sc;
      carry += __shfl_sync(kFull, sc, 31);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += hx;
  }
  return true;
}

// The step's test on the four values of mini block t: bits k of the result
// = row 32k + lane passes (and, with kGid, its group-id contribution added).
// kOp 0..4 = probe modes, 5 = group key, 6 = RANGE, 7 = NOTRANGE, 8 = IN.
template <int kOp, bool kGid>
__device__ __forceinline__ uint32_t staged_mb_test(const DevStep& S, const uint8_t* stab, const uint32_t (&v)[4],
                                                   uint32_t live, uint32_t (&gid)[4], unsigned int* status) {
  uint32_t keep = 0;
  if (kOp < PM_OPEN) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      keep |= uint32_t(probe_direct<kOp, kGid>(S, stab, v[k], true, gid[k])) << k;
  } else if (kOp == PM_OPEN) {
    const bool in_smem = S.smem_width != 0;
    const uint2* tab = in_smem ? reinterpret_cast<const uint2*>(stab + S.smem_off) : static_cast<const uint2*>(S.ht);
    const uint32_t mask = S.ht_mask;
    uint32_t h[4], pend = 0, pay[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = fmix32(v[k]) & mask;
      pay[k] = 0;
      if (((live >> k) & 1u) && int32_t(v[k]) != kEmptyKey) pend |= 1u << k;
    }
    for (uint32_t n = 0; pend && n <= mask; ++n) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((pend >> k) & 1u)) continue;
        const uint2 e = in_smem ? tab[h[k]] : __ldg(tab + h[k]);
        if (e.x == v[k]) {
          keep |= 1u << k;
          pay[k] = e.y;
          pend &= ~(1u << k);
        } else if (int32_t(e.x) == kEmptyKey) {
          pend &= ~(1u << k);
        } else {
          h[k] = (h[k] + 1) & mask;
        }
      }
    }
    if (pend) atomicOr(status, S_INTERNAL);
    if (kGid) {
#pragma unroll
      for (int k = 0; k < 4; ++k) gid[k] += (pay[k] & 0xffffu) * S.mul0 + (pay[k] >> 16) * S.mul1;
    }
  } else if (kOp == 5) {
    if (kGid) {
#pragma unroll
      for (int k = 0; k < 4; ++k) gid[k] += v[k] * S.key_mul;
    }
    keep = 15u;
  } else if (kOp == 6 || kOp == 7) {
    const uint32_t lo = uint32_t(S.lo), span = uint32_t(S.hi) - uint32_t(S.lo);
#pragma unroll
    for (int k = 0; k < 4; ++k) keep |= uint32_t(((v[k] - lo) <= span) != (kOp == 7)) << k;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool hit = false;
      for (int i = 0; i < S.nin; ++i) hit |= (int32_t(v[k]) == S.in[i]);
      keep |= uint32_t(hit && S.kind == ST_IN) << k;
    }
  }
  return keep;
}

template <bool kDelta, bool kGid, int kOp>
__device__ __forceinline__ void staged_dense(const DevStep& S, const TileHdr& Hd, TileState& T, const uint8_t* stab,
                                             StagedPay sp, int lane, unsigned int* status) {
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    uint32_t v[4];
    if (!staged_mb_decode<kDelta>(Hd, S.col, t, T.alive, sp, lane, v, status)) continue;
    const uint32_t live = (T.alive >> (4 * t)) & 15u;
    const uint32_t keep = staged_mb_test<kOp, kGid>(S, stab, v, live, T.gid[t], status);
    T.alive &= ~((~keep & 15u) << (4 * t));
  }
}

template <bool kHost, bool kDelta, bool kGid = true, bool kStaged = false>
__device__ __forceinline__ void dense_step_t(const DevQuery& Q, const DevStep& S, const PageState& P,
                                             const TileHdr& Hd, TileState& T, const uint8_t* stab, int lane,
                                             unsigned int* status, StagedPay sp = StagedPay{nullptr, 0, 0}) {
  // mini blocks that cannot hold a passing value are neither loaded nor decoded
  const uint32_t pruned = pruned_mbs<kDelta>(Hd, S.col, S.zlo, S.zhi, lane);
#pragma unroll
  for (int t = 0; t < TB; ++t)
    if ((pruned >> t) & 1u) T.alive &= ~(15u << (4 * t));
  if constexpr (kStaged) {
    switch (S.kind) {
      case ST_PROBE:
        switch (probe_mode(S)) {
          case PM_S1: staged_dense<kDelta, kGid, PM_S1>(S, Hd, T, stab, sp, lane, status); break;
          case PM_S2: staged_dense<kDelta, kGid, PM_S2>(S, Hd, T, stab, sp, lane, status); break;
          case PM_S4: staged_dense<kDelta, kGid, PM_S4>(S, Hd, T, stab, sp, lane, status); break;
          case PM_GDIRECT:
            if (kGid && (S.mul0 | S.mul1)) staged_dense<kDelta, kGid, PM_GDIRECT>(S, Hd, T, stab, sp, lane, status);
            else staged_dense<kDelta, false, PM_GDIRECT>(S, Hd, T, stab, sp, lane, status);
            break;
          default: staged_dense<kDelta, kGid, PM_OPEN>(S, Hd, T, stab, sp, lane, status); break;
        }
        return;
      case ST_KEY:
        if (kGid) staged_dense<kDelta, kGid, 5>(S, Hd, T, stab, sp, lane, status);
        else if (lane == 0) atomicOr(status, S_INTERNAL);  // the kernel routes group-key first steps to kGid
        return;
      case ST_RANGE: staged_dense<kDelta, kGid, 6>(S, Hd, T, stab, sp, lane, status); return;
      case ST_NOTRANGE: staged_dense<kDelta, kGid, 7>(S, Hd, T, stab, sp, lane, status); return;
      default: staged_dense<kDelta, kGid, 8>(S, Hd, T, stab, sp, lane, status); return;
    }
  }
  uint32_t v[TB][4];
  uint32_t anym;
  decode_t<kHost, kDelta, kStaged>(Q, S.col, P, Hd, T.alive, lane, v, anym, status, sp);
  switch (S.kind) {
    case ST_PROBE:
      switch (probe_mode(S)) {
        case PM_S1: dense_probe<PM_S1, kGid>(S, stab, v, anym, T, status); break;
        case PM_S2: dense_probe<PM_S2, kGid>(S, stab, v, anym, T, status); break;
        case PM_S4: dense_probe<PM_S4, kGid>(S, stab, v, anym, T, status); break;
        case PM_GDIRECT:
          if (S.ht_kind == HT_RANK) {
            if (kGid && (S.mul0 | S.mul1)) dense_probe_rank<kGid>(S, v, anym, T);
            else dense_probe_rank<false>(S, v, anym, T);
          } else if (kGid && (S.mul0 | S.mul1)) {
            dense_probe<PM_GDIRECT, kGid>(S, stab, v, anym, T, status);
          } else {
            dense_probe<PM_GDIRECT, false>(S, stab, v, anym, T, status);
          }
          break;
        default: dense_probe<PM_OPEN, kGid>(S, stab, v, anym, T, status); break;
      }
      return;
    case ST_KEY:
      if (kGid) {
#pragma unroll
        for (int t = 0; t < TB; ++t)
#pragma unroll
          for (int k = 0; k < 4; ++k) T.gid[t][k] += v[t][k] * S.key_mul;
      } else if (lane == 0) {
        atomicOr(status, S_INTERNAL);  // the kernel routes group-key first steps to kGid
      }
      return;
    case ST_RANGE:
    case ST_NOTRANGE: {
      const bool neg = S.kind == ST_NOTRANGE;
      // lo <= x <= hi  <=>  (x - lo) <= (hi - lo) as unsigned
      const uint32_t lo = uint32_t(S.lo), span = uint32_t(S.hi) - uint32_t(S.lo);
      uint32_t keep = 0;
#pragma unroll
      for (int t = 0; t < TB; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) keep |= uint32_t(((v[t][k] - lo) <= span) != neg) << (4 * t + k);
      T.alive &= keep;
      return;
    }
    default: {  // IN (FALSE compiles to IN with an empty list)
      uint32_t keep = 0;
#pragma unroll
      for (int t = 0; t < TB; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          bool hit = false;
          for (int i = 0; i < S.nin; ++i) hit |= (int32_t(v[t][k]) == S.in[i]);
          keep |= uint32_t(hit) << (4 * t + k);
        }
      T.alive &= S.kind == ST_IN ? keep : 0u;
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// Survivor lists.  After the first step the live rows of a tile are compacted
// (ballot + popc rank, the warp's selection vector) into a per-warp list in
// shared memory, entry = row-in-tile | group id << kRowBits, and every later
// step, and the aggregation, runs over the list with one survivor per lane,
// so the warp's issue slots follow the surviving rows instead of all rows.
// ---------------------------------------------------------------------------
constexpr uint32_t kTileRows = kMB * TB;
// A warp's list collects the survivors of several consecutive tiles of one
// page (a segment of at most 2^kRowBits rows) before the later steps run,
// so their rounds of 32 are full even when few rows survive per tile.
constexpr uint32_t kRowBits = 12;
constexpr uint32_t kSegMbs = (1u << kRowBits) / kMB;  // mini blocks per segment (16)
constexpr uint32_t kListCap = 1024;                    // entries per warp list
constexpr int kListUnroll = 1;  // survivor rounds whose loads are issued together (measured best at 1)
static_assert(kTileRows <= (1u << kRowBits), "row index field too narrow");
static_assert(kListCap >= kTileRows, "a list must hold one tile");
static_assert(kListBytesPerWarp == kListCap * 4, "the host's per-warp shared-memory figure");
static_assert(kSegMbs <= 32, "segment mini blocks must fit a 32-bit mask");

// Dense step s of a tile (or none): live bits and group-id contributions.
// The step's kind, table and codec are resolved here, once per tile.
// kGid = false compiles the step without group-id contributions (for a
// first step that adds none: a predicate, or a probe of a table no group key
// reads), which keeps the sixteen per-row group ids out of registers.
// kStaged: the step's packed words come from the warp's staging ring (sp);
// only integer first steps are staged.
template <bool kHost, bool kText = true, bool kGid = true, bool kStaged = false>
__device__ __forceinline__ void tile_dense_step(const DevQuery& Q, uint32_t s, const PageState& P, const TileHdr& Hd,
                                                TileState& T, const uint8_t* stab, int lane, unsigned int* status,
                                                StagedPay sp = StagedPay{nullptr, 0, 0}) {
  if (s >= Q.nsteps) return;
  const DevStep& S = Q.steps[s];
  if (S.kind == ST_ALL) return;  // every row passes; its column is never read
  if (S.kind == ST_PREFIX || S.kind == ST_CONTAINS || S.kind == ST_LIKE) {
    if (!kStaged) tile_prefix<kHost, kText>(Q, S, P, Hd, T, lane, status, stab);
    else if (lane == 0) atomicOr(status, S_INTERNAL);
  } else if (Q.cols[S.col].codec == C_DELTA) {
    dense_step_t<kHost, true, kGid, kStaged>(Q, S, P, Hd, T, stab, lane, status, sp);
  } else {
    dense_step_t<kHost, false, kGid, kStaged>(Q, S, P, Hd, T, stab, lane, status, sp);
  }
}

// Whether step S adds a group-id contribution when it runs densely.
__device__ __forceinline__ bool step_adds_gid(const DevStep& S) {
  return S.kind == ST_KEY || (S.kind == ST_PROBE && (S.mul0 | S.mul1) != 0);
}

// Appends the tile's live rows to the warp's list after its first n0
// entries; row_base = the tile's first row within the list's segment.
// Returns the list length.  Each lane counts its live rows, a warp exclusive
// scan of the counts gives the lane's first slot, and the lane writes its
// rows there in (t, k) order (the list's order is free: later steps and the
// aggregation visit every entry once, whatever its position).
template <bool kGid = true>
__device__ __forceinline__ uint32_t tile_compact(const TileState& T, uint32_t* list, uint32_t n0, uint32_t row_base,
                                                 int lane) {
  const uint32_t cnt = __popc(T.alive);
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  uint32_t pos = n0 + incl - cnt;
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if ((T.alive >> (4 * t + k)) & 1u) {
        list[pos] = (row_base + uint32_t(t * kMB + k * 32 + lane)) | (kGid ? T.gid[t][k] << kRowBits : 0u);
        ++pos;
      }
  __syncwarp();
  return n0 + total;
}

// Value of FOR/DICT column c at row r of the list's segment (mini blocks
// seg_mb.. of the page): the mini block's header (an L1 hit: the tile's
// headers were just loaded) and one bit field of its packed payload (two
// words when the field straddles them).
template <bool kHost>
__device__ __forceinline__ uint32_t point_value(const DevQuery& Q, int c, const PageState& P, uint32_t seg_mb,
                                                uint32_t r, bool valid) {
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  if (!valid) return 0u;
  const uint32_t codec = Q.cols[c].codec;
  const uint2 h = ld_u2<kHost>(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(seg_mb + (r >> 7)) * 8));
  const uint32_t bw = tmin<uint32_t>(h.y & 0xffu, 32u);
  uint32_t x = 0;
  if (bw != 0) {
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(codec, P.prow));
    const uint32_t bit = (r & (kMB - 1)) * bw;
    const uint32_t* p = pay + (h.y >> 8) + (bit >> 5);
    const uint32_t sh = bit & 31u;
    const uint32_t lo = ld_u32<kHost>(p);
    const uint32_t hi = sh + bw > 32 ? ld_u32<kHost>(p + 1) : 0u;
    x = __funnelshift_r(lo, hi, sh);
    if (bw < 32) x &= (1u << bw) - 1u;
  }
  return h.x + x;
}

// Dense decode of one mini block mb of column c whose header is read from
// the page (lane i < bw loads word k*bw + i): v[k] = value of row 32k + lane.
template <bool kHost>
__device__ __forceinline__ void mb_decode_at(const DevQuery& Q, int c, const uint8_t* pg, const PageState& P,
                                             uint32_t mb, int lane, uint32_t (&v)[4], unsigned int* status) {
  const uint32_t codec = Q.cols[c].codec;
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + payload_offset(codec, P.prow));
  uint32_t first, dmin = 0, wob;
  if (codec == C_DELTA) {
    const uint4 h = ld_u4<kHost>(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(mb) * 16));
    first = h.x;
    dmin = h.y;
    wob = h.z;
  } else {
    const uint2 h = ld_u2<kHost>(reinterpret_cast<const uint2*>(pg + kPageHdr + uint64_t(mb) * 8));
    first = h.x;
    wob = h.y;
  }
  uint32_t bw = wob & 0xffu;
  if (bw > 32) {
    if (lane == 0) atomicOr(status, S_CORRUPT);
    bw = 0;
  }
  const bool ld = uint32_t(lane) < bw;
  const uint32_t* w = pay + (wob >> 8) + lane;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = unpack_lane(ld ? ld_u32<kHost>(w + uint32_t(k) * bw) : 0u, bw, lane);
  if (codec == C_DELTA) {
    // x_j = first + sum_{i<=j} (dmin + p_i), modulo 2^32
    uint32_t carry = first;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t sc = warp_incl_scan(v[k] + dmin, lane);
      v[k] = carry + sc;
      carry += __shfl_sync(kFull, sc, 31);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += first;
  }
}

// Value of any integer column at segment row r.  A DELTA mini block with
// bit width 0 holds one repeated value (every delta is dmin = 0: the runs of
// equal keys of a sorted load), which its header gives directly.  Other
// DELTA mini blocks need the prefix sum of their deltas, so each one holding
// a row of the round is decoded densely and the lanes pick their rows with
// shuffles.
template <bool kHost>
__device__ __forceinline__ uint32_t row_value(const DevQuery& Q, int c, const PageState& P, uint32_t seg_mb,
                                              uint32_t r, bool valid, int lane, unsigned int* status) {
  if (Q.cols[c].codec != C_DELTA) return point_value<kHost>(Q, c, P, seg_mb, r, valid);
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  uint32_t out = 0;
  bool dense = false;
  if (valid) {
    const uint4 h = ld_u4<kHost>(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(seg_mb + (r >> 7)) * 16));
    if ((h.z & 0xffu) == 0 && h.y == 0) out = h.x;  // constant mini block
    else dense = true;
  }
  uint32_t need = __reduce_or_sync(kFull, dense ? 1u << (r >> 7) : 0u);
  while (need) {
    const uint32_t t = uint32_t(__ffs(need) - 1);
    need &= need - 1;
    uint32_t v[4];
    mb_decode_at<kHost>(Q, c, pg, P, seg_mb + t, lane, v, status);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = __shfl_sync(kFull, v[k], int(r & 31));
      if (dense && (r >> 5) == t * 4 + uint32_t(k)) out = x;
    }
  }
  return out;
}

// PREFIX / CONTAINS on a list: lengths and starts of the round's mini
// blocks are decoded densely and gathered per lane, then each string is
// matched (kText = false: raw PREFIX only, as for tile_prefix).
template <bool kHost, bool kText = true>
__device__ __forceinline__ bool row_prefix(const DevQuery& Q, const DevStep& S, const PageState& P,
                                           uint32_t seg_mb, uint32_t r, bool valid, int lane,
                                           unsigned int* status, const uint8_t* stab) {
  const int c = S.col;
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  const uint32_t* starts = reinterpret_cast<const uint32_t*>(pg + kPageHdr + uint64_t(P.nmb_page) * 8);
  uint32_t need = __reduce_or_sync(kFull, valid ? 1u << (r >> 7) : 0u);
  uint32_t my_len = 0, my_start = 0;
  while (need) {
    const uint32_t t = uint32_t(__ffs(need) - 1);
    need &= need - 1;
    uint32_t len[4], st[4];
    mb_decode_at<kHost>(Q, c, pg, P, seg_mb + t, lane, len, status);
    excl_scan128(len, lane, st);
    const uint32_t mb_start = ld_u32<kHost>(starts + seg_mb + t);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t l = __shfl_sync(kFull, len[k], int(r & 31));
      const uint32_t s0 = __shfl_sync(kFull, st[k], int(r & 31));
      if (valid && (r >> 5) == t * 4 + uint32_t(k)) {
        my_len = l;
        my_start = mb_start + s0;
      }
    }
  }
  const uint8_t* bytes = pg + __shfl_sync(kFull, P.extra, c) + my_start;
  const int4* sym = Q.cols[c].codec == C_FSST ? Q.cols[c].sym : nullptr;
  if constexpr (kText) {
    const uint8_t* tab = sym != nullptr && S.smem_width ? stab + S.smem_off : nullptr;
    return valid && string_match<kHost>(S, bytes, my_len, sym, tab);
  } else {
    if (!valid) return false;
    if (S.kind != ST_PREFIX || sym != nullptr) {
      atomicOr(status, S_INTERNAL);
      return false;
    }
    if (my_len < S.plen) return false;
    for (uint32_t i = 0; i < S.plen; ++i)
      if (ld_u8<kHost>(bytes + i) != S.pfx[i]) return false;
    return true;
  }
}

// Join probe of one key; on a hit adds the join's group-id contribution.
template <int kMode>
__device__ __forceinline__ bool row_probe(const DevStep& S, const uint8_t* stab, uint32_t key, bool valid,
                                          uint32_t& gid, unsigned int* status) {
  if (kMode != PM_OPEN) return probe_direct<kMode>(S, stab, key, valid, gid);
  if (!valid || int32_t(key) == kEmptyKey) return false;
  const uint2* tab = S.smem_width ? reinterpret_cast<const uint2*>(stab + S.smem_off) : static_cast<const uint2*>(S.ht);
  uint32_t pay;
  if (!ht_probe(tab, S.ht_mask, int32_t(key), &pay, status)) return false;
  gid += (pay & 0xffffu) * S.mul0 + (pay >> 16) * S.mul1;
  return true;
}

// One later step over a warp's list for a FOR/DICT column, specialised on the
// operation: kOp 0..4 = probe modes, 5 = group key, 6 = RANGE, 7 = NOTRANGE,
// 8 = IN / FALSE.  Returns the new list length.
template <bool kHost, int kOp>
__device__ __forceinline__ uint32_t list_step_t(const DevQuery& Q, const DevStep& S, const PageState& P,
                                                uint32_t seg_mb, uint32_t* list, uint32_t n, const uint8_t* stab,
                                                int lane, unsigned int* status) {
  // Rounds of 32 survivors are taken kListUnroll at a time: their entries
  // and packed values are all loaded before any is used, so the warp keeps
  // that many independent loads in flight.  Compacted entries are written
  // only after the group's entries were read, never ahead of them.
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t out = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += 32 * kListUnroll) {
    uint32_t r[kListUnroll], gid[kListUnroll], v[kListUnroll];
    bool valid[kListUnroll];
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) {
      valid[u] = i0 + 32u * u + lane < n;
      const uint32_t e = valid[u] ? list[i0 + 32u * u + lane] : 0u;
      r[u] = e & ((1u << kRowBits) - 1u);
      gid[u] = e >> kRowBits;
    }
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) v[u] = point_value<kHost>(Q, S.col, P, seg_mb, r[u], valid[u]);
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kListUnroll; ++u) {
      bool keep;
      if (kOp <= PM_OPEN) {
        keep = row_probe<kOp>(S, stab, v[u], valid[u], gid[u], status);
      } else if (kOp == 5) {
        gid[u] += v[u] * S.key_mul;
        keep = valid[u];
      } else if (kOp == 6 || kOp == 7) {
        keep = valid[u] && (((v[u] - uint32_t(S.lo)) <= uint32_t(S.hi) - uint32_t(S.lo)) != (kOp == 7));
      } else {
        keep = valid[u] && step_pred(S, int32_t(v[u]));
      }
      const uint32_t m = __ballot_sync(kFull, keep);
      if (keep) list[out + __popc(m & lt)] = r[u] | (gid[u] << kRowBits);
      out += __popc(m);
    }
  }
  __syncwarp();
  return out;
}

// Value of a FOR64 column (Sec. 4.1, 64-bit GPU-FOR) at segment row r: the
// mini block's 16-byte header {base, word offset, bit width} and the row's
// field at bit (r % 128) * bw of the mini block's 64-bit words, read through
// a 128-bit window (the second word only when the field crosses into it).
// Other integer columns are read as int32 and sign-extended.  Warp-uniform
// call (c is uniform); lanes with !valid return 0.
template <bool kHost>
__device__ __forceinline__ long long value64(const DevQuery& Q, int c, const PageState& P, uint32_t seg_mb,
                                             uint32_t r, bool valid, int lane, unsigned int* status) {
  if (Q.cols[c].codec != C_FOR64) return (long long)int32_t(row_value<kHost>(Q, c, P, seg_mb, r, valid, lane, status));
  const uint8_t* pg = reinterpret_cast<const uint8_t*>(__shfl_sync(kFull, P.pg, c));
  if (!valid) return 0;
  const uint4 h = ld_u4<kHost>(reinterpret_cast<const uint4*>(pg + kPageHdr + uint64_t(seg_mb + (r >> 7)) * 16));
  const unsigned long long base = (unsigned long long)h.x | ((unsigned long long)h.y << 32);
  const uint32_t bw = tmin<uint32_t>(h.w, 64u);  // validated at load
  unsigned long long x = 0;
  if (bw != 0) {
    const uint2* pay = reinterpret_cast<const uint2*>(pg + payload_offset(C_FOR64, P.prow));
    const uint32_t bit = (r & (kMB - 1)) * bw;
    const uint2* p = pay + h.z + (bit >> 6);
    const uint32_t sh = bit & 63u;
    const uint2 lo = ld_u2<kHost>(p);
    x = ((unsigned long long)lo.x | ((unsigned long long)lo.y << 32)) >> sh;
    if (sh + bw > 64) {
      const uint2 hi = ld_u2<kHost>(p + 1);
      x |= ((unsigned long long)hi.x | ((unsigned long long)hi.y << 32)) << (64 - sh);
    }
    if (bw < 64) x &= (1ull << bw) - 1ull;
  }
  return (long long)(base + x);
}

// A later step on a DELTA column, a string step (dense decode of the
// round's mini blocks) or a 64-bit range over a FOR64 column (one field per
// survivor, value64); kept out of line.
template <bool kHost, bool kText = true>
__device__ __noinline__ uint32_t list_step_generic(const DevQuery& Q, const DevStep& S, const PageState& P,
                                                   uint32_t seg_mb, uint32_t* list, uint32_t n,
                                                   const uint8_t* stab, int lane, unsigned int* status) {
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t out = 0;
  for (uint32_t i0 = 0; i0 < n; i0 += 32) {
    const bool valid = i0 + lane < n;
    const uint32_t e = valid ? list[i0 + lane] : 0u;
    const uint32_t r = e & ((1u << kRowBits) - 1u);
    uint32_t gid = e >> kRowBits;
    bool keep;
    if (S.kind == ST_PREFIX || S.kind == ST_CONTAINS || S.kind == ST_LIKE) {
      keep = row_prefix<kHost, kText>(Q, S, P, seg_mb, r, valid, lane, status, stab);
    } else if (is_step64(S.kind)) {
      const int64_t x = value64<kHost>(Q, S.col, P, seg_mb, r, valid, lane, status);
      const bool in = step_bound64(S.in, 0) <= x && x <= step_bound64(S.in, 1);
      keep = valid && (in != (S.kind == ST_NOTRANGE64));
    } else {
      const uint32_t v = row_value<kHost>(Q, S.col, P, seg_mb, r, valid, lane, status);
      if (S.kind == ST_PROBE) {
        switch (probe_mode(S)) {
          case PM_S1: keep = row_probe<PM_S1>(S, stab, v, valid, gid, status); break;
          case PM_S2: keep = row_probe<PM_S2>(S, stab, v, valid, gid, status); break;
          case PM_S4: keep = row_probe<PM_S4>(S, stab, v, valid, gid, status); break;
          case PM_GDIRECT: keep = row_probe<PM_GDIRECT>(S, stab, v, valid, gid, status); break;
          default: keep = row_probe<PM_OPEN>(S, stab, v, valid, gid, status); break;
        }
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
  return out;
}

// Steps first.. of the query over the warp's list; returns the list length.  Each
// step is resolved to its specialised loop once, outside the loop.
template <bool kHost, bool kText = true>
__device__ __forceinline__ uint32_t list_steps(const DevQuery& Q, const PageState& P, uint32_t seg_mb,
                                               uint32_t* list, uint32_t n, const uint8_t* stab, int lane,
                                               unsigned int* status, uint32_t first = 1) {
  for (uint32_t s = first; s < Q.nsteps && n != 0; ++s) {
    const DevStep& S = Q.steps[s];
    if (S.kind == ST_PREFIX || S.kind == ST_CONTAINS || S.kind == ST_LIKE || Q.cols[S.col].codec == C_DELTA ||
        is_step64(S.kind)) {
      n = list_step_generic<kHost, kText>(Q, S, P, seg_mb, list, n, stab, lane, status);
      continue;
    }
    switch (S.kind) {
      case ST_PROBE:
        switch (probe_mode(S)) {
          case PM_S1: n = list_step_t<kHost, PM_S1>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
          case PM_S2: n = list_step_t<kHost, PM_S2>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
          case PM_S4: n = list_step_t<kHost, PM_S4>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
          case PM_GDIRECT: n = list_step_t<kHost, PM_GDIRECT>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
          default: n = list_step_t<kHost, PM_OPEN>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
        }
        break;
      case ST_KEY: n = list_step_t<kHost, 5>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
      case ST_RANGE: n = list_step_t<kHost, 6>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
      case ST_NOTRANGE: n = list_step_t<kHost, 7>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
      default: n = list_step_t<kHost, 8>(Q, S, P, seg_mb, list, n, stab, lane, status); break;
    }
  }
  return n;
}

}  // namespace dpf

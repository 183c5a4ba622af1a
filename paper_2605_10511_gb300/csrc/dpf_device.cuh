// Device helpers shared by the library's kernels: mini block header parsing,
// warp-cooperative unpacking of 128-value mini blocks (four values per lane,
// lane l holding rows l, l+32, l+64, l+96 as in the four-values-per-thread
// decompression of Sec. 3.2), delta and length prefix sums, predicates and
// hash probes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dpf_internal.h"

namespace dpf {

constexpr unsigned kFull = 0xffffffffu;

template <class T>
__host__ __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <class T>
__host__ __device__ __forceinline__ T tmax(T a, T b) { return a < b ? b : a; }

// MurmurHash3's 32-bit finaliser: a published bijective mixer.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

struct MbHdr {
  int32_t base;   // FOR base (FOR/DICT/STR lengths) or dmin (DELTA)
  int32_t first;  // DELTA first value
  uint32_t bw;
  uint32_t woff;  // payload offset in 32-bit words
};

__device__ __forceinline__ MbHdr parse_hdr(uint4 h, uint32_t codec) {
  MbHdr m;
  if (codec == C_DELTA) {
    m.first = int32_t(h.x);
    m.base = int32_t(h.y);
    m.bw = h.z & 0xffu;
    m.woff = h.z >> 8;
  } else {
    m.first = 0;
    m.base = int32_t(h.x);
    m.bw = h.y & 0xffu;
    m.woff = h.y >> 8;
  }
  return m;
}

// Loads of compressed bytes.  Both device-resident and host-resident
// (mapped pinned) columns are immutable while a kernel runs, so both use
// the read-only path: full-width vector loads that the host link serves in
// whole lines.  (kHost selects the kernel instantiation for host-resident
// pages; the loads are the same.)
template <bool kHost>
__device__ __forceinline__ uint32_t ld_u32(const uint32_t* p) {
  return __ldg(p);
}
template <bool kHost>
__device__ __forceinline__ uint2 ld_u2(const uint2* p) {
  return __ldg(p);
}
template <bool kHost>
__device__ __forceinline__ uint4 ld_u4(const uint4* p) {
  return __ldg(p);
}
template <bool kHost>
__device__ __forceinline__ uint8_t ld_u8(const uint8_t* p) {
  return __ldg(p);
}

// Bits [lane*bw, lane*bw + bw) of the bw words w_k held one per lane
// (lane i holds word k*bw + i): one of the 32 values of group k.
__device__ __forceinline__ uint32_t unpack_lane(uint32_t wk, uint32_t bw, int lane) {
  const uint32_t bit = uint32_t(lane) * bw;
  const int src = int(bit >> 5);
  const uint32_t lo = __shfl_sync(kFull, wk, src);
  const uint32_t hi = __shfl_sync(kFull, wk, (src + 1) & 31);
  const uint32_t v = __funnelshift_r(lo, hi, bit & 31u);
  return bw >= 32 ? v : (v & ((1u << bw) - 1u));
}

// Inclusive warp prefix sum (mod 2^32).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// Decodes the 128 values of one mini block held in w[0..3] (lane i holds
// payload word k*bw + i of group k) into v[k] = value of row 32k + lane.
// FOR/DICT/STR-lengths: base + field.  DELTA: first + sum_{i<=j}(dmin + p_i).
__device__ __forceinline__ void decode_mb(const uint32_t (&w)[4], const MbHdr& h, uint32_t codec,
                                          int lane, uint32_t (&v)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = unpack_lane(w[k], h.bw, lane) + uint32_t(h.base);
  if (codec == C_DELTA) {
    uint32_t carry = uint32_t(h.first);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t s = warp_incl_scan(v[k], lane);
      v[k] = carry + s;
      carry += __shfl_sync(kFull, s, 31);
    }
  }
}

// Exclusive prefix of lengths over the 128 rows of a mini block, in row
// order (row 32k + lane): start offset of each string inside the mini block.
__device__ __forceinline__ void excl_scan128(const uint32_t (&len)[4], int lane,
                                             uint32_t (&start)[4]) {
  uint32_t carry = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t s = warp_incl_scan(len[k], lane);
    start[k] = carry + s - len[k];
    carry += __shfl_sync(kFull, s, 31);
  }
}

__device__ __forceinline__ bool step_pred(const DevStep& S, int32_t x) {
  switch (S.kind) {
    case ST_RANGE: return S.lo <= x && x <= S.hi;
    case ST_NOTRANGE: return !(S.lo <= x && x <= S.hi);
    case ST_IN: {
      bool hit = false;
      for (int i = 0; i < S.nin; ++i) hit |= (x == S.in[i]);
      return hit;
    }
    case ST_FALSE: return false;
    default: return true;
  }
}

// A rank-directory table: one 16-byte word per 64 keys of the range,
// {presence bits of keys 0-31, of keys 32-63, present keys before the word,
// present keys before its key 32}, then the present keys' payloads in key
// order.  Key offset off's bits live in 32-bit word rank_bits_word(off) of
// the directory and its running count two words later.
__device__ __forceinline__ uint32_t rank_bits_word(uint32_t off) {
  const uint32_t q = off >> 5;
  return (q >> 1) * 4u + (q & 1u);
}

// Payload of key kmin + off (off < krange) in a rank-directory table, or
// kAbsent: the key's presence bit, then the payload at the half word's
// running count plus the set bits below the key's.
__device__ __forceinline__ uint32_t rank_entry(const void* tab, uint32_t krange, uint32_t off) {
  const uint32_t* dw = static_cast<const uint32_t*>(tab);
  const uint32_t wi = rank_bits_word(off), bb = off & 31u;
  const uint32_t bits = __ldg(dw + wi);
  if (!((bits >> bb) & 1u)) return kAbsent;
  const uint32_t* pay = dw + 4 * ((uint64_t(krange) + 63) >> 6);
  return __ldg(pay + __ldg(dw + wi + 2) + uint32_t(__popc(bits & ((1u << bb) - 1u))));
}

// Bounded linear probe of an open-addressing table of capacity mask+1.
// Returns true and the payload on a hit; a probe that meets neither the key
// nor an empty slot within capacity steps sets S_INTERNAL.
__device__ __forceinline__ bool ht_probe(const uint2* tab, uint32_t mask, int32_t key,
                                         uint32_t* payload, unsigned int* status) {
  uint32_t h = fmix32(uint32_t(key)) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint2 s = tab[h];
    if (int32_t(s.x) == key) {
      *payload = s.y;
      return true;
    }
    if (int32_t(s.x) == kEmptyKey) return false;
    h = (h + 1) & mask;
  }
  atomicOr(status, S_INTERNAL);
  return false;
}

}  // namespace dpf

// Host-side loader: type-specific compression into the page format
// (Sec. 4.2 data loader; Sec. 3.4.1 GPU-FOR mini blocks; Sec. 3.4.2
// variable-length pages and the RID index; Sec. 4.1 integer decompression
// formats).  Pages are independent, so they are planned and written by a
// pool of host threads in two passes: sizes first, then bytes at their
// prefix-summed offsets (the two-pass loading of Sec. 4.2, in memory).
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "dpf_internal.h"
#include "host_common.h"

namespace dpf {
namespace {

struct MbPlan {
  int32_t base;     // FOR base, or DELTA dmin
  int32_t first;    // DELTA first value
  uint32_t bw;
  uint32_t word_off;
};

struct PagePlan {
  uint32_t rows, nmb, payload_off, extra_off;
  uint64_t bytes, str_bytes;
  std::vector<MbPlan> mb;
  std::vector<uint32_t> str_start;
};

inline uint32_t width_of(uint32_t span) { return span == 0 ? 0u : 32u - __builtin_clz(span); }

// Packs n32 = 128 values q[j] (already offset by the base) of width bw into
// 4*bw words, value j at bit j*bw, LSB first.
void pack128(const uint32_t* q, uint32_t bw, uint32_t* out) {
  std::memset(out, 0, size_t(4) * bw * 4);
  if (bw == 0) return;
  for (uint32_t j = 0; j < kMB; ++j) {
    const uint64_t bit = uint64_t(j) * bw;
    const uint32_t w = uint32_t(bit >> 5), s = uint32_t(bit & 31);
    out[w] |= q[j] << s;
    if (s + bw > 32) out[w + 1] |= q[j] >> (32 - s);
  }
}

// Values of mini block m of page p after the codec's transform:
// FOR/DICT -> value (or code), DELTA -> wrapped difference with the previous row.
struct IntSource {
  uint32_t codec;
  const int32_t* v;          // raw values (FOR, DELTA)
  const uint32_t* codes;     // DICT ranks
  int32_t at(uint64_t r) const { return codec == C_DICT ? int32_t(codes[r]) : v[r]; }
};

void plan_int_page(const IntSource& src, uint32_t codec, uint64_t r0, uint32_t rows, PagePlan& pp) {
  pp.rows = rows;
  pp.nmb = (rows + kMB - 1) / kMB;
  pp.mb.resize(pp.nmb);
  pp.payload_off = payload_offset(codec, rows);
  uint32_t words = 0;
  for (uint32_t m = 0; m < pp.nmb; ++m) {
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + rows - a));
    int64_t lo, hi;
    MbPlan& mp = pp.mb[m];
    if (codec == C_DELTA) {
      lo = hi = 0;  // d_0 = 0
      for (uint32_t j = 1; j < cnt; ++j) {
        const int64_t d = int32_t(uint32_t(src.at(a + j)) - uint32_t(src.at(a + j - 1)));
        lo = std::min(lo, d);
        hi = std::max(hi, d);
      }
      mp.first = src.at(a);
    } else {
      lo = hi = src.at(a);
      for (uint32_t j = 1; j < cnt; ++j) {
        const int64_t x = src.at(a + j);
        lo = std::min(lo, x);
        hi = std::max(hi, x);
      }
      mp.first = 0;
    }
    mp.base = int32_t(lo);
    mp.bw = width_of(uint32_t(uint64_t(hi - lo)));
    mp.word_off = words;
    words += 4 * mp.bw;
  }
  pp.extra_off = 0;
  pp.str_bytes = 0;
  pp.bytes = align16(uint64_t(pp.payload_off) + uint64_t(words) * 4);
}

void write_int_page(const IntSource& src, uint32_t codec, uint64_t r0, const PagePlan& pp,
                    uint8_t* pg) {
  std::memset(pg, 0, pp.bytes);
  const uint32_t hdr[4] = {kMagic | (codec << 24), pp.rows, pp.payload_off, 0};
  std::memcpy(pg, hdr, sizeof hdr);
  uint32_t* pay = reinterpret_cast<uint32_t*>(pg + pp.payload_off);
  uint32_t q[kMB];
  for (uint32_t m = 0; m < pp.nmb; ++m) {
    const MbPlan& mp = pp.mb[m];
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + pp.rows - a));
    for (uint32_t j = 0; j < kMB; ++j) {
      if (j >= cnt) { q[j] = 0; continue; }
      uint32_t t;
      if (codec == C_DELTA)
        t = j == 0 ? 0u : uint32_t(src.at(a + j)) - uint32_t(src.at(a + j - 1));
      else
        t = uint32_t(src.at(a + j));
      q[j] = t - uint32_t(mp.base);
    }
    pack128(q, mp.bw, pay + mp.word_off);
    uint8_t* h = pg + kPageHdr + uint64_t(m) * mb_hdr_bytes(codec);
    const uint32_t wob = (mp.word_off << 8) | mp.bw;
    if (codec == C_DELTA) {
      const uint32_t w[4] = {uint32_t(mp.first), uint32_t(mp.base), wob, 0};
      std::memcpy(h, w, 16);
    } else {
      const uint32_t w[2] = {uint32_t(mp.base), wob};
      std::memcpy(h, w, 8);
    }
  }
}

// 64-bit frame of reference (Sec. 4.1, GPU-FOR extended to BIGINT): 64-bit
// bases, fields of bw <= 64 bits at bit j*bw of a stream of 64-bit words.
struct Mb64 {
  int64_t base;
  uint32_t bw, word_off;
};

inline uint32_t width_of64(uint64_t span) { return span == 0 ? 0u : 64u - uint32_t(__builtin_clzll(span)); }

// Packs 128 fields q[j] (already offset by the base) of width bw into 2*bw
// words, field j at bit j*bw, LSB first; a field crossing a word boundary
// continues at bit 0 of the next word.
void pack128_64(const uint64_t* q, uint32_t bw, uint64_t* out) {
  std::memset(out, 0, size_t(2) * bw * 8);
  if (bw == 0) return;
  for (uint32_t j = 0; j < kMB; ++j) {
    const uint64_t bit = uint64_t(j) * bw;
    const uint32_t w = uint32_t(bit >> 6), s = uint32_t(bit & 63);
    out[w] |= q[j] << s;
    if (s + bw > 64) out[w + 1] |= q[j] >> (64 - s);
  }
}

// Mini block plans of one FOR64 page; returns the page's byte size.
uint64_t plan_for64_page(const int64_t* v, uint64_t r0, uint32_t rows, std::vector<Mb64>& mb) {
  const uint32_t nmb = (rows + kMB - 1) / kMB;
  mb.resize(nmb);
  uint64_t words = 0;
  for (uint32_t m = 0; m < nmb; ++m) {
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + rows - a));
    int64_t lo = v[a], hi = v[a];
    for (uint32_t j = 1; j < cnt; ++j) {
      lo = std::min(lo, v[a + j]);
      hi = std::max(hi, v[a + j]);
    }
    mb[m].base = lo;
    mb[m].bw = width_of64(uint64_t(hi) - uint64_t(lo));
    mb[m].word_off = uint32_t(words);
    words += 2ull * mb[m].bw;
  }
  return align16(uint64_t(payload_offset(C_FOR64, rows)) + words * 8);
}

void write_for64_page(const int64_t* v, uint64_t r0, uint32_t rows, const std::vector<Mb64>& mb,
                      uint64_t bytes, uint8_t* pg) {
  std::memset(pg, 0, bytes);
  const uint32_t poff = payload_offset(C_FOR64, rows);
  const uint32_t hdr[4] = {kMagic | (uint32_t(C_FOR64) << 24), rows, poff, 0};
  std::memcpy(pg, hdr, sizeof hdr);
  uint64_t* pay = reinterpret_cast<uint64_t*>(pg + poff);
  uint64_t q[kMB];
  for (uint32_t m = 0; m < uint32_t(mb.size()); ++m) {
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + rows - a));
    for (uint32_t j = 0; j < kMB; ++j) q[j] = j < cnt ? uint64_t(v[a + j]) - uint64_t(mb[m].base) : 0u;
    pack128_64(q, mb[m].bw, pay + mb[m].word_off);
    uint8_t* h = pg + kPageHdr + uint64_t(m) * 16;
    std::memcpy(h, &mb[m].base, 8);
    std::memcpy(h + 8, &mb[m].word_off, 4);
    std::memcpy(h + 12, &mb[m].bw, 4);
  }
}

void plan_str_page(const uint64_t* offs, uint64_t r0, uint32_t rows, PagePlan& pp, bool* bad) {
  // (STR and FSST pages share this layout)
  pp.rows = rows;
  pp.nmb = (rows + kMB - 1) / kMB;
  pp.mb.resize(pp.nmb);
  pp.str_start.resize(pp.nmb);
  pp.payload_off = payload_offset(C_STR, rows);
  uint32_t words = 0;
  uint64_t bytes = 0;
  for (uint32_t m = 0; m < pp.nmb; ++m) {
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + rows - a));
    if (bytes > 0xffffffffull) *bad = true;
    pp.str_start[m] = uint32_t(bytes);
    uint64_t lo = ~0ull, hi = 0;
    for (uint32_t j = 0; j < cnt; ++j) {
      const uint64_t len = offs[a + j + 1] - offs[a + j];
      if (len > 0x7fffffffull) *bad = true;
      lo = std::min(lo, len);
      hi = std::max(hi, len);
      bytes += len;
    }
    MbPlan& mp = pp.mb[m];
    mp.base = int32_t(lo);
    mp.first = 0;
    mp.bw = width_of(uint32_t(hi - lo));
    mp.word_off = words;
    words += 4 * mp.bw;
  }
  if (bytes > 0xffffffffull) *bad = true;
  pp.extra_off = uint32_t(align16(uint64_t(pp.payload_off) + uint64_t(words) * 4));
  pp.str_bytes = bytes;
  pp.bytes = align16(uint64_t(pp.extra_off) + bytes);
}

void write_str_page(uint32_t codec, const uint8_t* data, const uint64_t* offs, uint64_t r0, const PagePlan& pp,
                    uint8_t* pg) {
  std::memset(pg, 0, pp.extra_off);
  const uint32_t hdr[4] = {kMagic | (codec << 24), pp.rows, pp.payload_off, pp.extra_off};
  std::memcpy(pg, hdr, sizeof hdr);
  uint32_t* pay = reinterpret_cast<uint32_t*>(pg + pp.payload_off);
  uint32_t q[kMB];
  for (uint32_t m = 0; m < pp.nmb; ++m) {
    const MbPlan& mp = pp.mb[m];
    const uint64_t a = r0 + uint64_t(m) * kMB;
    const uint32_t cnt = std::min<uint32_t>(kMB, uint32_t(r0 + pp.rows - a));
    for (uint32_t j = 0; j < kMB; ++j)
      q[j] = j < cnt ? uint32_t(offs[a + j + 1] - offs[a + j]) - uint32_t(mp.base) : 0u;
    pack128(q, mp.bw, pay + mp.word_off);
    const uint32_t w[2] = {uint32_t(mp.base), (mp.word_off << 8) | mp.bw};
    std::memcpy(pg + kPageHdr + uint64_t(m) * 8, w, 8);
    std::memcpy(pg + kPageHdr + uint64_t(pp.nmb) * 8 + uint64_t(m) * 4, &pp.str_start[m], 4);
  }
  std::memcpy(pg + pp.extra_off, data + offs[r0], pp.str_bytes);
  std::memset(pg + pp.extra_off + pp.str_bytes, 0, pp.bytes - pp.extra_off - pp.str_bytes);
}

// ---------------------------------------------------------------- FSST
// Symbol table of the FSST string codec (Sec. 3.4.2, Sec. 4.1), built with
// the construction of Boncz, Neumann and Leis (VLDB 2020): up to 255 symbols
// of 1..8 bytes; an encoded string is a sequence of codes, c < nsym for
// symbol c and 255 (escape) followed by a literal byte.  Over five
// generations a sample of the strings is parsed greedily with the current
// table; every token (a symbol, or an escaped byte) and every concatenation
// of two consecutive tokens of at most 8 bytes is counted, and the 255
// candidates of largest count x length form the next table.  Encoding is
// greedy: the longest symbol matching at each position.
struct FsstTable {
  uint32_t n = 0;
  uint8_t len[kFsstMaxSymbols];
  uint64_t sym[kFsstMaxSymbols];             // bytes, little endian
  std::vector<uint8_t> by_first[256];         // codes starting with a byte, longest first
  void index() {
    for (auto& v : by_first) v.clear();
    for (uint32_t c = 0; c < n; ++c) by_first[sym[c] & 0xffu].push_back(uint8_t(c));
    for (auto& v : by_first)
      std::stable_sort(v.begin(), v.end(), [&](uint8_t a, uint8_t b) { return len[a] > len[b]; });
  }
  // Longest symbol at s[0..avail): its code, or -1.
  int match(const uint8_t* s, uint64_t avail) const;
};

inline uint64_t load_bytes(const uint8_t* p, uint32_t len) {
  uint64_t x = 0;
  std::memcpy(&x, p, len);
  return x;
}

int FsstTable::match(const uint8_t* s, uint64_t avail) const {
  for (uint8_t c : by_first[s[0]]) {
    const uint32_t l = len[c];
    if (l <= avail && load_bytes(s, l) == sym[c]) return c;
  }
  return -1;
}

// A token as a 64-bit key: its bytes in the low 56 bits... does not fit 8
// bytes, so tokens are kept as (bytes, length) pairs in one 128-bit word.
struct TokKey {
  uint64_t bytes;
  uint32_t len;
  bool operator==(const TokKey& o) const { return bytes == o.bytes && len == o.len; }
};
struct TokHash {
  size_t operator()(const TokKey& k) const { return std::hash<uint64_t>()(k.bytes * 0x9e3779b97f4a7c15ull ^ k.len); }
};

FsstTable fsst_choose(const uint8_t* data, const uint64_t* offs, uint64_t n) {
  FsstTable t;
  t.index();
  const uint64_t sample = std::min<uint64_t>(n, 16384);
  for (int gen = 0; gen < 5; ++gen) {
    std::unordered_map<TokKey, uint64_t, TokHash> count;
    for (uint64_t r = 0; r < sample; ++r) {
      const uint8_t* s = data + offs[r];
      const uint64_t L = offs[r + 1] - offs[r];
      TokKey prev{0, 0};
      for (uint64_t i = 0; i < L;) {
        const int c = t.match(s + i, L - i);
        const uint32_t l = c >= 0 ? t.len[c] : 1u;
        const TokKey tok{load_bytes(s + i, l), l};
        ++count[tok];
        if (prev.len && prev.len + l <= 8) ++count[TokKey{prev.bytes | (tok.bytes << (8 * prev.len)), prev.len + l}];
        prev = tok;
        i += l;
      }
    }
    std::vector<std::pair<TokKey, uint64_t>> cand(count.begin(), count.end());
    std::sort(cand.begin(), cand.end(), [](const std::pair<TokKey, uint64_t>& a, const std::pair<TokKey, uint64_t>& b) {
      const uint64_t ga = a.second * a.first.len, gb = b.second * b.first.len;
      if (ga != gb) return ga > gb;
      if (a.first.len != b.first.len) return a.first.len < b.first.len;
      return a.first.bytes < b.first.bytes;
    });
    t.n = 0;
    for (const auto& c : cand) {
      if (t.n == kFsstMaxSymbols) break;
      t.len[t.n] = uint8_t(c.first.len);
      t.sym[t.n] = c.first.bytes;
      ++t.n;
    }
    t.index();
  }
  return t;
}

// Encodes one string; returns the encoded length (out: room for 2 * len).
uint64_t fsst_encode(const FsstTable& t, const uint8_t* s, uint64_t len, uint8_t* out) {
  uint64_t o = 0;
  for (uint64_t i = 0; i < len;) {
    const int code = t.match(s + i, len - i);
    if (code >= 0) {
      out[o++] = uint8_t(code);
      i += t.len[code];
    } else {
      out[o++] = uint8_t(kFsstEscape);
      out[o++] = s[i++];
    }
  }
  return o;
}

// Sorted distinct values (at most `limit`, else returns false).
bool distinct_sorted(const int32_t* v, uint64_t n, std::vector<int32_t>& out, size_t limit) {
  const unsigned T = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(host_threads(), n / 65536 + 1));
  std::vector<std::vector<int32_t>> part(T);
  bool over = false;
  parallel_for(T, [&](uint64_t t) {
    const uint64_t a = n * t / T, b = n * (t + 1) / T;
    std::vector<int32_t>& p = part[t];
    // collect distinct values of the slice incrementally to bound memory
    std::vector<int32_t> buf;
    buf.reserve(std::min<uint64_t>(b - a, 1u << 16));
    for (uint64_t r = a; r < b; ++r) {
      buf.push_back(v[r]);
      if (buf.size() == (1u << 16) || r + 1 == b) {
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        std::vector<int32_t> merged;
        merged.reserve(p.size() + buf.size());
        std::set_union(p.begin(), p.end(), buf.begin(), buf.end(), std::back_inserter(merged));
        p.swap(merged);
        buf.clear();
        if (p.size() > limit) { over = true; return; }
      }
    }
  });
  if (over) return false;
  out.clear();
  for (auto& p : part) {
    std::vector<int32_t> merged;
    std::set_union(out.begin(), out.end(), p.begin(), p.end(), std::back_inserter(merged));
    out.swap(merged);
    if (out.size() > limit) return false;
  }
  return true;
}

}  // namespace
}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_encode_column(const dpf_column_desc* desc, const void* values,
                                        const uint64_t* str_offsets, uint64_t nrows, uint8_t* out,
                                        uint64_t cap, uint64_t* page_off, uint64_t* row_prefix,
                                        int32_t* dict, uint64_t dict_cap, uint64_t* dict_n,
                                        uint64_t* size_out) {
  if (!desc) return fail(DPF_EINVAL, "encode: desc is NULL");
  const uint32_t codec = uint32_t(desc->codec);
  const uint32_t P = desc->page_rows ? desc->page_rows : kDefaultPageRows;
  if (nrows == 0) return fail(DPF_EINVAL, "encode: nrows must be > 0");
  if (P % kMB != 0 || P > kMaxPageRows) return fail(DPF_EINVAL, "encode: page_rows %u not a multiple of 128 in [128, 2^20]", P);
  if (codec < C_FOR || codec > C_FOR64) return fail(DPF_EINVAL, "encode: unknown codec %u", codec);
  if (!values && !is_str_codec(codec)) return fail(DPF_EINVAL, "encode: values is NULL");
  if (is_str_codec(codec) && !str_offsets) return fail(DPF_EINVAL, "encode: STR/FSST needs str_offsets");
  if (!page_off || !row_prefix || !size_out) return fail(DPF_EINVAL, "encode: page_off/row_prefix/size_out NULL");

  const uint64_t npages = (nrows + P - 1) / P;
  if (codec == C_FOR64) {
    const int64_t* v = static_cast<const int64_t*>(values);
    std::vector<std::vector<Mb64>> mbs(npages);
    std::vector<uint64_t> bytes(npages);
    parallel_for(npages, [&](uint64_t p) {
      bytes[p] = plan_for64_page(v, p * P, uint32_t(std::min<uint64_t>(P, nrows - p * P)), mbs[p]);
    });
    uint64_t off = 0;
    for (uint64_t p = 0; p < npages; ++p) {
      page_off[p] = off;
      row_prefix[p] = std::min<uint64_t>(nrows, (p + 1) * P);
      off += bytes[p];
    }
    page_off[npages] = off;
    *size_out = off;
    if (dict_n) *dict_n = 0;
    if (!out) return DPF_OK;
    if (cap < off) return fail(DPF_ETRUNC, "encode: cap %llu < %llu", (unsigned long long)cap, (unsigned long long)off);
    parallel_for(npages, [&](uint64_t p) {
      write_for64_page(v, p * P, uint32_t(std::min<uint64_t>(P, nrows - p * P)), mbs[p], bytes[p], out + page_off[p]);
    });
    return DPF_OK;
  }
  std::vector<PagePlan> plans(npages);
  std::vector<uint32_t> codes;
  std::vector<int32_t> dvals;
  IntSource src{codec, static_cast<const int32_t*>(values), nullptr};
  // FSST: the strings encoded with the column's symbol table, then written as
  // STR pages of the encoded bytes
  std::vector<uint8_t> fenc;
  std::vector<uint64_t> foff;
  const uint8_t* sbytes = static_cast<const uint8_t*>(values);
  const uint64_t* soffs = str_offsets;
  if (is_str_codec(codec)) {
    for (uint64_t r = 0; r < nrows; ++r)
      if (str_offsets[r + 1] < str_offsets[r]) return fail(DPF_EINVAL, "encode: str_offsets not monotone at row %llu", (unsigned long long)r);
    if (str_offsets[nrows] != str_offsets[0] && !values) return fail(DPF_EINVAL, "encode: values is NULL");
  }
  if (codec == C_FSST) {
    const uint8_t* raw = sbytes;
    const FsstTable t = fsst_choose(raw, str_offsets, nrows);
    if (dict_n) *dict_n = 3ull * t.n;
    if (dict) {
      if (dict_cap < 3ull * t.n) return fail(DPF_ETRUNC, "encode: dict_cap %llu < %u", (unsigned long long)dict_cap, 3 * t.n);
      for (uint32_t c = 0; c < t.n; ++c) {
        dict[3 * c] = int32_t(uint32_t(t.sym[c]));
        dict[3 * c + 1] = int32_t(uint32_t(t.sym[c] >> 32));
        dict[3 * c + 2] = int32_t(t.len[c]);
      }
    }
    // encode page by page in parallel into per-page buffers, then join
    std::vector<std::vector<uint8_t>> pe(npages);
    std::vector<std::vector<uint64_t>> po(npages);
    parallel_for(npages, [&](uint64_t p) {
      const uint64_t r0 = p * P, r1 = std::min<uint64_t>(nrows, r0 + P);
      pe[p].resize(2 * (str_offsets[r1] - str_offsets[r0]) + 1);
      po[p].assign(r1 - r0, 0);
      uint64_t o = 0;
      for (uint64_t r = r0; r < r1; ++r) {
        o += fsst_encode(t, raw + str_offsets[r], str_offsets[r + 1] - str_offsets[r], pe[p].data() + o);
        po[p][r - r0] = o;
      }
      pe[p].resize(o);
    });
    foff.assign(nrows + 1, 0);
    uint64_t total = 0;
    for (uint64_t p = 0; p < npages; ++p) {
      for (uint64_t i = 0; i < po[p].size(); ++i) foff[p * P + i + 1] = total + po[p][i];
      total += pe[p].size();
    }
    fenc.resize(std::max<uint64_t>(total, 1));
    parallel_for(npages, [&](uint64_t p) {
      if (!pe[p].empty()) std::memcpy(fenc.data() + foff[p * P], pe[p].data(), pe[p].size());
    });
    sbytes = fenc.data();
    soffs = foff.data();
  }
  if (is_str_codec(codec)) {
    bool bad = false;
    parallel_for(npages, [&](uint64_t p) {
      const uint64_t r0 = p * P;
      plan_str_page(soffs, r0, uint32_t(std::min<uint64_t>(P, nrows - r0)), plans[p], &bad);
    });
    if (bad) return fail(DPF_EINVAL, "encode: a page holds >= 4 GiB of string bytes or a string >= 2 GiB");
  } else {
    if (codec == C_DICT) {
      if (!distinct_sorted(src.v, nrows, dvals, 65536)) return fail(DPF_EINVAL, "encode: DICT column has more than 65536 distinct values");
      codes.resize(nrows);
      parallel_for((nrows + 65535) / 65536, [&](uint64_t b) {
        const uint64_t a = b * 65536, e = std::min<uint64_t>(nrows, a + 65536);
        for (uint64_t r = a; r < e; ++r)
          codes[r] = uint32_t(std::lower_bound(dvals.begin(), dvals.end(), src.v[r]) - dvals.begin());
      });
      src.codes = codes.data();
      if (dict_n) *dict_n = dvals.size();
      if (dict) {
        if (dict_cap < dvals.size()) return fail(DPF_ETRUNC, "encode: dict_cap %llu < %zu", (unsigned long long)dict_cap, dvals.size());
        std::copy(dvals.begin(), dvals.end(), dict);
      }
    }
    parallel_for(npages, [&](uint64_t p) {
      const uint64_t r0 = p * P;
      plan_int_page(src, codec, r0, uint32_t(std::min<uint64_t>(P, nrows - r0)), plans[p]);
    });
  }
  uint64_t off = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    page_off[p] = off;
    row_prefix[p] = std::min<uint64_t>(nrows, (p + 1) * P);
    off += plans[p].bytes;
  }
  page_off[npages] = off;
  *size_out = off;
  if (!out) return DPF_OK;
  if (cap < off) return fail(DPF_ETRUNC, "encode: cap %llu < %llu", (unsigned long long)cap, (unsigned long long)off);
  parallel_for(npages, [&](uint64_t p) {
    if (is_str_codec(codec))
      write_str_page(codec, sbytes, soffs, p * P, plans[p], out + page_off[p]);
    else
      write_int_page(src, codec, p * P, plans[p], out + page_off[p]);
  });
  return DPF_OK;
}

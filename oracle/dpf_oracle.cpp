// Reference oracle for the fused query path -- TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may
// load this library.  It shares no code, header or constant generator with
// the CUDA library: every layout constant below is restated here from the
// storage-format definition (Sec. 3.4.1 fixed-length page layout with
// mini blocks carrying a frame-of-reference base, a bit width and a byte
// offset; Sec. 3.4.2 variable-length pages with a RID index that is a
// prefix sum of per-page record counts; Sec. 4.1 integer decompression,
// 32-bit GPU-FOR and its 64-bit extension for BIGINT columns;
// Sec. 4.2 data-loader metadata: page offsets and per-page row prefix).
//
// What it computes (Sec. 3.1, Kernels #1-#3): an exact relational result
//   SELECT keys, COUNT(*), aggs FROM fact JOIN dims WHERE conj GROUP BY keys
// with inner equi-joins on unique dimension keys (a dimension may itself be
// joined with further dimensions before it is built: a chain such as
// LINEITEM -> ORDERS -> CUSTOMER) and every aggregate held
// in int64 after sign-extending the int32 inputs (Sec. 4.3, DECIMAL stored
// as 32-bit and processed as 64-bit).  The evaluator is deliberately plain:
// it decodes whole columns first (page by page, mini block by mini block,
// bit by bit), then walks the fact rows one at a time, looks dimension keys
// up in std::unordered_map built from the rows that pass the dimension
// predicates (the build side of Kernel #1), and accumulates groups in a
// std::map ordered by the key tuple (the record-format result of Kernel #3).
// orc_query_threads runs the same row walk on several host threads over
// disjoint page ranges and adds their group records together (int64
// addition modulo 2^64, so the records are those of the one-thread walk);
// it exists to evaluate tables of 2^28-2^30 rows in the tests in minutes.
//
// Parity status of every function here: pinned by the tests under
// tests/test_oracle_*.py (hand-worked golden bytes, encode/decode round
// trips on edge cases, an independent numpy evaluator on small tables,
// invariants).  None is "parity unpinned".

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

// <thread> defines errno's EINVAL macro; the status names below are this file's own.
#undef EINVAL

namespace {

// ---- storage-format constants, restated from the format definition ----
constexpr uint32_t kMiniBlock = 128;           // values per mini block
constexpr uint32_t kPageHeaderBytes = 16;      // magic|codec, nrows, payload_off, extra_off
constexpr uint32_t kMagic = 0x00465044u;       // 'D' 'P' 'F' in the low three bytes
enum Codec : uint32_t { FOR = 1, DELTA = 2, DICT = 3, STR = 4, FSST = 5, FOR64 = 6 };

enum Status : int64_t {
  OK = 0,
  EINVAL = -1,
  ETRUNC = -7,
  EDUPKEY = -4,
  ECORRUPT = -9,
};

uint64_t align16(uint64_t x) { return (x + 15u) & ~uint64_t(15); }

// Bits needed to hold span = max - min (0 when all values are equal).
uint32_t bits_for_span(uint64_t span) {
  uint32_t b = 0;
  while (b < 64 && (span >> b) != 0) ++b;
  return b;
}

uint32_t mb_header_bytes(uint32_t codec) { return codec == DELTA ? 16u : 8u; }

// Writes p[0..127] at bit j*bw (bit b of the stream is bit b%32 of word b/32),
// one bit at a time.
void pack_bits(const uint32_t* p, uint32_t bw, uint32_t* words) {
  for (uint32_t w = 0; w < 4 * bw; ++w) words[w] = 0;
  for (uint32_t j = 0; j < kMiniBlock; ++j)
    for (uint32_t b = 0; b < bw; ++b)
      if ((p[j] >> b) & 1u) {
        uint64_t bit = uint64_t(j) * bw + b;
        words[bit / 32] |= 1u << (bit % 32);
      }
}

// Reads the bw-bit field j, one bit at a time.
uint32_t unpack_bits(const uint32_t* words, uint32_t bw, uint32_t j) {
  uint32_t v = 0;
  for (uint32_t b = 0; b < bw; ++b) {
    uint64_t bit = uint64_t(j) * bw + b;
    v |= ((words[bit / 32] >> (bit % 32)) & 1u) << b;
  }
  return v;
}

struct PageLayout {
  uint32_t nrows, nmb, hdr_bytes, payload_off, payload_bytes, extra_off;
  uint64_t extra_bytes, page_bytes;
};

// Frame-of-reference plan of one mini block of already-transformed values
// q[0..cnt): returns (base, bw).  Missing trailing rows repeat the base.
void for_plan(const int64_t* q, uint32_t cnt, int64_t* base, uint32_t* bw) {
  int64_t mn = q[0], mx = q[0];
  for (uint32_t j = 1; j < cnt; ++j) { mn = std::min(mn, q[j]); mx = std::max(mx, q[j]); }
  *base = mn;
  *bw = bits_for_span(uint64_t(mx - mn));
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Integer column encoding (FOR, DELTA, DICT codes).
//
// values[0..n) -> blob.  page_off[npages+1] receives each page's byte offset
// (the last entry is the blob size); row_prefix[npages] receives the RID
// index (cumulative rows up to and including page i).  For DICT, dict_out
// receives the sorted distinct values (capacity dict_cap) and *dict_n their
// count.  With out == nullptr only the sizes are computed.  Returns the blob
// size in bytes or a negative status.
// ---------------------------------------------------------------------------
int64_t orc_encode_int(uint32_t codec, const int32_t* values, uint64_t n, uint32_t page_rows,
                       uint8_t* out, uint64_t cap, uint64_t* page_off, uint64_t* row_prefix,
                       int32_t* dict_out, uint64_t dict_cap, uint64_t* dict_n) {
  if (n == 0 || page_rows == 0 || page_rows % kMiniBlock != 0 || page_rows > (1u << 20))
    return EINVAL;
  if (codec != FOR && codec != DELTA && codec != DICT) return EINVAL;

  // DICT: codes are ranks in the sorted distinct values.
  std::vector<int32_t> dict;
  std::vector<int64_t> src(n);
  if (codec == DICT) {
    dict.assign(values, values + n);
    std::sort(dict.begin(), dict.end());
    dict.erase(std::unique(dict.begin(), dict.end()), dict.end());
    if (dict.size() > 65536) return EINVAL;
    for (uint64_t r = 0; r < n; ++r)
      src[r] = std::lower_bound(dict.begin(), dict.end(), values[r]) - dict.begin();
    if (dict_n) *dict_n = dict.size();
    if (dict_out) {
      if (dict.size() > dict_cap) return ETRUNC;
      std::copy(dict.begin(), dict.end(), dict_out);
    }
  } else {
    for (uint64_t r = 0; r < n; ++r) src[r] = values[r];
  }

  const uint64_t npages = (n + page_rows - 1) / page_rows;
  uint64_t off = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint64_t r0 = p * page_rows;
    const uint32_t rows = uint32_t(std::min<uint64_t>(page_rows, n - r0));
    const uint32_t nmb = (rows + kMiniBlock - 1) / kMiniBlock;
    const uint32_t hb = mb_header_bytes(codec);
    const uint32_t payload_off = uint32_t(align16(kPageHeaderBytes + uint64_t(nmb) * hb));
    // plan every mini block
    std::vector<int64_t> q(kMiniBlock);
    std::vector<uint32_t> bws(nmb);
    std::vector<int64_t> bases(nmb), firsts(nmb);
    uint64_t words = 0;
    for (uint32_t m = 0; m < nmb; ++m) {
      const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
      const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
      if (codec == DELTA) {
        // d_0 = 0, d_j = x_j - x_{j-1} taken as a wrapped 32-bit signed difference
        q[0] = 0;
        for (uint32_t j = 1; j < cnt; ++j)
          q[j] = int32_t(uint32_t(src[a + j]) - uint32_t(src[a + j - 1]));
        firsts[m] = src[a];
      } else {
        for (uint32_t j = 0; j < cnt; ++j) q[j] = src[a + j];
      }
      for_plan(q.data(), cnt, &bases[m], &bws[m]);
      if (bws[m] > 32) return EINVAL;
      words += 4ull * bws[m];
    }
    if (words >= (1ull << 24)) return EINVAL;
    const uint64_t page_bytes = align16(payload_off + words * 4);
    if (page_off) page_off[p] = off;
    if (row_prefix) row_prefix[p] = r0 + rows;
    if (out) {
      if (off + page_bytes > cap) return ETRUNC;
      uint8_t* pg = out + off;
      std::memset(pg, 0, page_bytes);
      const uint32_t hdr[4] = {kMagic | (codec << 24), rows, payload_off, 0};
      std::memcpy(pg, hdr, sizeof hdr);
      uint32_t* pay = reinterpret_cast<uint32_t*>(pg + payload_off);
      uint32_t woff = 0;
      std::vector<uint32_t> pk(kMiniBlock);
      for (uint32_t m = 0; m < nmb; ++m) {
        const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
        const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
        for (uint32_t j = 0; j < kMiniBlock; ++j) {
          int64_t t;
          if (j >= cnt) t = bases[m];                               // padding: offset 0
          else if (codec == DELTA) t = j == 0 ? 0 : int32_t(uint32_t(src[a + j]) - uint32_t(src[a + j - 1]));
          else t = src[a + j];
          pk[j] = uint32_t(uint64_t(t - bases[m]));
        }
        pack_bits(pk.data(), bws[m], pay + woff);
        uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * mb_header_bytes(codec);
        const uint32_t wob = (woff << 8) | bws[m];
        if (codec == DELTA) {
          const int32_t f = int32_t(firsts[m]), dmin = int32_t(bases[m]);
          const uint32_t zero = 0;
          std::memcpy(h, &f, 4);
          std::memcpy(h + 4, &dmin, 4);
          std::memcpy(h + 8, &wob, 4);
          std::memcpy(h + 12, &zero, 4);
        } else {
          const int32_t b = int32_t(bases[m]);
          std::memcpy(h, &b, 4);
          std::memcpy(h + 4, &wob, 4);
        }
        woff += 4 * bws[m];
      }
    }
    off += page_bytes;
  }
  if (page_off) page_off[npages] = off;
  return int64_t(off);
}

// Decodes every row of an integer column.  For DICT the result is the
// dictionary value (codes are looked up in dict[0..dict_n)).  Returns 0 or a
// negative status (ECORRUPT on a bad page header or mini block header).
int64_t orc_decode_int(uint32_t codec, const uint8_t* blob, const uint64_t* page_off,
                       uint64_t npages, uint64_t n, uint32_t page_rows, const int32_t* dict,
                       uint64_t dict_n, int32_t* out) {
  uint64_t r = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint8_t* pg = blob + page_off[p];
    uint32_t hdr[4];
    std::memcpy(hdr, pg, sizeof hdr);
    if (hdr[0] != (kMagic | (codec << 24))) return ECORRUPT;
    const uint32_t rows = hdr[1];
    if (rows == 0 || rows > page_rows || r + rows > n) return ECORRUPT;
    const uint32_t nmb = (rows + kMiniBlock - 1) / kMiniBlock;
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + hdr[2]);
    const uint64_t pay_words = (page_off[p + 1] - page_off[p] - hdr[2]) / 4;
    for (uint32_t m = 0; m < nmb; ++m) {
      const uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * mb_header_bytes(codec);
      int32_t base, first = 0;
      uint32_t wob;
      if (codec == DELTA) {
        std::memcpy(&first, h, 4);
        std::memcpy(&base, h + 4, 4);
        std::memcpy(&wob, h + 8, 4);
      } else {
        std::memcpy(&base, h, 4);
        std::memcpy(&wob, h + 4, 4);
      }
      const uint32_t bw = wob & 0xffu, woff = wob >> 8;
      if (bw > 32 || uint64_t(woff) + 4ull * bw > pay_words) return ECORRUPT;
      const uint32_t cnt = std::min<uint32_t>(kMiniBlock, rows - m * kMiniBlock);
      uint32_t running = uint32_t(first);
      for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t f = unpack_bits(pay + woff, bw, j);
        int32_t v;
        if (codec == DELTA) {
          // v_j = first + sum_{i<=j} (dmin + p_i), all modulo 2^32
          running += uint32_t(base) + f;
          v = int32_t(running);
        } else {
          v = int32_t(uint32_t(base) + f);
        }
        if (codec == DICT) {
          if (uint32_t(v) >= dict_n) return ECORRUPT;
          v = dict[uint32_t(v)];
        }
        out[r + j] = v;
      }
      r += cnt;
    }
  }
  return r == n ? OK : ECORRUPT;
}

// Row lookup through the RID index: binary search for the first page whose
// cumulative row count exceeds r, then decode that single value.
int64_t orc_decode_int_row(uint32_t codec, const uint8_t* blob, const uint64_t* page_off,
                           const uint64_t* row_prefix, uint64_t npages, const int32_t* dict,
                           uint64_t dict_n, uint64_t r, int32_t* out) {
  uint64_t lo = 0, hi = npages;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    if (row_prefix[mid] > r) hi = mid; else lo = mid + 1;
  }
  if (lo >= npages) return EINVAL;
  const uint64_t page_first = lo == 0 ? 0 : row_prefix[lo - 1];
  const uint8_t* pg = blob + page_off[lo];
  uint32_t hdr[4];
  std::memcpy(hdr, pg, sizeof hdr);
  if (hdr[0] != (kMagic | (codec << 24))) return ECORRUPT;
  const uint32_t i = uint32_t(r - page_first);
  const uint32_t m = i / kMiniBlock, j = i % kMiniBlock;
  const uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * mb_header_bytes(codec);
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + hdr[2]);
  int32_t base, first = 0;
  uint32_t wob;
  if (codec == DELTA) {
    std::memcpy(&first, h, 4);
    std::memcpy(&base, h + 4, 4);
    std::memcpy(&wob, h + 8, 4);
  } else {
    std::memcpy(&base, h, 4);
    std::memcpy(&wob, h + 4, 4);
  }
  const uint32_t bw = wob & 0xffu, woff = wob >> 8;
  if (bw > 32) return ECORRUPT;
  uint32_t v;
  if (codec == DELTA) {
    v = uint32_t(first);
    for (uint32_t k = 0; k <= j; ++k) v += uint32_t(base) + unpack_bits(pay + woff, bw, k);
  } else {
    v = uint32_t(base) + unpack_bits(pay + woff, bw, j);
  }
  if (codec == DICT) {
    if (v >= dict_n) return ECORRUPT;
    v = uint32_t(dict[v]);
  }
  *out = int32_t(v);
  return OK;
}

// ---------------------------------------------------------------------------
// 64-bit frame of reference (Sec. 4.1: GPU-FOR extended to BIGINT with 64-bit
// reference values and bit positions taken modulo 64).  Per page: the page
// header, one 16-byte header per mini block {base: int64, word offset: u32
// counted in 8-byte words from the payload start, bit width: u32 in 0..64},
// then the payload of 64-bit words.  Field j of a mini block holds x_j - base
// (modulo 2^64) at bits [j*bw, (j+1)*bw) of its 2*bw words (128 fields of bw
// bits fill exactly 2*bw words, so every mini block starts on a word), bit b
// of the stream being bit b%64 of word b/64.
// ---------------------------------------------------------------------------
static void pack_bits64(const uint64_t* f, uint32_t bw, uint64_t* words) {
  for (uint32_t w = 0; w < 2 * bw; ++w) words[w] = 0;
  for (uint32_t j = 0; j < kMiniBlock; ++j)
    for (uint32_t b = 0; b < bw; ++b)
      if ((f[j] >> b) & 1u) {
        const uint64_t bit = uint64_t(j) * bw + b;
        words[bit / 64] |= uint64_t(1) << (bit % 64);
      }
}

static uint64_t unpack_bits64(const uint64_t* words, uint32_t bw, uint32_t j) {
  uint64_t v = 0;
  for (uint32_t b = 0; b < bw; ++b) {
    const uint64_t bit = uint64_t(j) * bw + b;
    v |= ((words[bit / 64] >> (bit % 64)) & 1u) << b;
  }
  return v;
}

int64_t orc_encode_for64(const int64_t* values, uint64_t n, uint32_t page_rows, uint8_t* out, uint64_t cap,
                         uint64_t* page_off, uint64_t* row_prefix) {
  if (n == 0 || page_rows == 0 || page_rows % kMiniBlock != 0 || page_rows > (1u << 20)) return EINVAL;
  const uint64_t npages = (n + page_rows - 1) / page_rows;
  uint64_t off = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint64_t r0 = p * page_rows;
    const uint32_t rows = uint32_t(std::min<uint64_t>(page_rows, n - r0));
    const uint32_t nmb = (rows + kMiniBlock - 1) / kMiniBlock;
    const uint32_t payload_off = uint32_t(align16(kPageHeaderBytes + uint64_t(nmb) * 16));
    std::vector<int64_t> bases(nmb);
    std::vector<uint32_t> bws(nmb);
    uint64_t words = 0;
    for (uint32_t m = 0; m < nmb; ++m) {
      const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
      const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
      int64_t mn = values[a], mx = values[a];
      for (uint32_t j = 1; j < cnt; ++j) { mn = std::min(mn, values[a + j]); mx = std::max(mx, values[a + j]); }
      bases[m] = mn;
      bws[m] = bits_for_span(uint64_t(mx) - uint64_t(mn));
      words += 2ull * bws[m];
    }
    if (words >= (1ull << 32)) return EINVAL;
    const uint64_t page_bytes = align16(payload_off + words * 8);
    if (page_off) page_off[p] = off;
    if (row_prefix) row_prefix[p] = r0 + rows;
    if (out) {
      if (off + page_bytes > cap) return ETRUNC;
      uint8_t* pg = out + off;
      std::memset(pg, 0, page_bytes);
      const uint32_t hdr[4] = {kMagic | (uint32_t(FOR64) << 24), rows, payload_off, 0};
      std::memcpy(pg, hdr, sizeof hdr);
      uint64_t* pay = reinterpret_cast<uint64_t*>(pg + payload_off);
      uint32_t woff = 0;
      std::vector<uint64_t> f(kMiniBlock);
      for (uint32_t m = 0; m < nmb; ++m) {
        const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
        const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
        for (uint32_t j = 0; j < kMiniBlock; ++j)   // padding rows: offset 0
          f[j] = j < cnt ? uint64_t(values[a + j]) - uint64_t(bases[m]) : 0;
        pack_bits64(f.data(), bws[m], pay + woff);
        uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * 16;
        std::memcpy(h, &bases[m], 8);
        std::memcpy(h + 8, &woff, 4);
        std::memcpy(h + 12, &bws[m], 4);
        woff += 2 * bws[m];
      }
    }
    off += page_bytes;
  }
  if (page_off) page_off[npages] = off;
  return int64_t(off);
}

// One value of a FOR64 page: mini block m, field j.  Returns false on a bad
// mini block header.
static bool for64_value(const uint8_t* pg, uint64_t pay_words, uint32_t m, uint32_t j, int64_t* v) {
  const uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * 16;
  int64_t base;
  uint32_t woff, bw, poff;
  std::memcpy(&base, h, 8);
  std::memcpy(&woff, h + 8, 4);
  std::memcpy(&bw, h + 12, 4);
  std::memcpy(&poff, pg + 8, 4);
  if (bw > 64 || uint64_t(woff) + 2ull * bw > pay_words) return false;
  const uint64_t* pay = reinterpret_cast<const uint64_t*>(pg + poff);
  *v = int64_t(uint64_t(base) + unpack_bits64(pay + woff, bw, j));
  return true;
}

int64_t orc_decode_for64(const uint8_t* blob, const uint64_t* page_off, uint64_t npages, uint64_t n,
                         uint32_t page_rows, int64_t* out) {
  uint64_t r = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint8_t* pg = blob + page_off[p];
    uint32_t hdr[4];
    std::memcpy(hdr, pg, sizeof hdr);
    if (hdr[0] != (kMagic | (uint32_t(FOR64) << 24))) return ECORRUPT;
    const uint32_t rows = hdr[1];
    if (rows == 0 || rows > page_rows || r + rows > n) return ECORRUPT;
    const uint64_t pay_words = (page_off[p + 1] - page_off[p] - hdr[2]) / 8;
    for (uint32_t i = 0; i < rows; ++i)
      if (!for64_value(pg, pay_words, i / kMiniBlock, i % kMiniBlock, out + r + i)) return ECORRUPT;
    r += rows;
  }
  return r == n ? OK : ECORRUPT;
}

// Row lookup through the RID index (binary search over the per-page row
// prefix, as for the 32-bit codecs).
int64_t orc_decode_for64_row(const uint8_t* blob, const uint64_t* page_off, const uint64_t* row_prefix,
                             uint64_t npages, uint64_t r, int64_t* out) {
  uint64_t lo = 0, hi = npages;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if (row_prefix[mid] > r) hi = mid; else lo = mid + 1;
  }
  if (lo >= npages) return EINVAL;
  const uint64_t i = r - (lo == 0 ? 0 : row_prefix[lo - 1]);
  const uint8_t* pg = blob + page_off[lo];
  uint32_t hdr[4];
  std::memcpy(hdr, pg, sizeof hdr);
  if (hdr[0] != (kMagic | (uint32_t(FOR64) << 24))) return ECORRUPT;
  const uint64_t pay_words = (page_off[lo + 1] - page_off[lo] - hdr[2]) / 8;
  return for64_value(pg, pay_words, uint32_t(i / kMiniBlock), uint32_t(i % kMiniBlock), out) ? OK : ECORRUPT;
}

// ---------------------------------------------------------------------------
// Variable-length strings (Sec. 3.4.2 with the offsets delta-coded): per page
// the string lengths are FOR-packed in mini blocks of 128, each mini block
// also records the byte offset of its first string inside the page's byte
// region, and the raw bytes follow.  offsets[0..n] are the caller's byte
// offsets into bytes (offsets[r+1] - offsets[r] = length of row r).
// ---------------------------------------------------------------------------
static int64_t encode_str_pages(uint32_t codec, const uint8_t* bytes, const uint64_t* offsets, uint64_t n,
                                uint32_t page_rows, uint8_t* out, uint64_t cap, uint64_t* page_off,
                                uint64_t* row_prefix) {
  if (n == 0 || page_rows == 0 || page_rows % kMiniBlock != 0 || page_rows > (1u << 20))
    return EINVAL;
  const uint64_t npages = (n + page_rows - 1) / page_rows;
  uint64_t off = 0;
  std::vector<int64_t> q(kMiniBlock);
  std::vector<uint32_t> pk(kMiniBlock);
  for (uint64_t p = 0; p < npages; ++p) {
    const uint64_t r0 = p * page_rows;
    const uint32_t rows = uint32_t(std::min<uint64_t>(page_rows, n - r0));
    const uint32_t nmb = (rows + kMiniBlock - 1) / kMiniBlock;
    const uint32_t payload_off = uint32_t(align16(kPageHeaderBytes + uint64_t(nmb) * 12));
    std::vector<uint32_t> bws(nmb), starts(nmb);
    std::vector<int64_t> bases(nmb);
    uint64_t words = 0, nbytes = 0;
    for (uint32_t m = 0; m < nmb; ++m) {
      const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
      const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
      if (nbytes >= (1ull << 32)) return EINVAL;
      starts[m] = uint32_t(nbytes);
      for (uint32_t j = 0; j < cnt; ++j) {
        const uint64_t len = offsets[a + j + 1] - offsets[a + j];
        if (len > 0x7fffffffu) return EINVAL;
        q[j] = int64_t(len);
        nbytes += len;
      }
      for_plan(q.data(), cnt, &bases[m], &bws[m]);
      words += 4ull * bws[m];
    }
    if (words >= (1ull << 24) || nbytes >= (1ull << 32)) return EINVAL;
    const uint32_t extra_off = uint32_t(align16(payload_off + words * 4));
    const uint64_t page_bytes = align16(extra_off + nbytes);
    if (page_off) page_off[p] = off;
    if (row_prefix) row_prefix[p] = r0 + rows;
    if (out) {
      if (off + page_bytes > cap) return ETRUNC;
      uint8_t* pg = out + off;
      std::memset(pg, 0, page_bytes);
      const uint32_t hdr[4] = {kMagic | (codec << 24), rows, payload_off, extra_off};
      std::memcpy(pg, hdr, sizeof hdr);
      uint32_t* pay = reinterpret_cast<uint32_t*>(pg + payload_off);
      uint32_t woff = 0;
      for (uint32_t m = 0; m < nmb; ++m) {
        const uint64_t a = r0 + uint64_t(m) * kMiniBlock;
        const uint32_t cnt = uint32_t(std::min<uint64_t>(kMiniBlock, r0 + rows - a));
        for (uint32_t j = 0; j < kMiniBlock; ++j) {
          const int64_t len = j < cnt ? int64_t(offsets[a + j + 1] - offsets[a + j]) : bases[m];
          pk[j] = uint32_t(uint64_t(len - bases[m]));
        }
        pack_bits(pk.data(), bws[m], pay + woff);
        uint8_t* h = pg + kPageHeaderBytes + uint64_t(m) * 8;
        const int32_t b = int32_t(bases[m]);
        const uint32_t wob = (woff << 8) | bws[m];
        std::memcpy(h, &b, 4);
        std::memcpy(h + 4, &wob, 4);
        std::memcpy(pg + kPageHeaderBytes + uint64_t(nmb) * 8 + uint64_t(m) * 4, &starts[m], 4);
        woff += 4 * bws[m];
      }
      std::memcpy(pg + extra_off, bytes + offsets[r0], offsets[r0 + rows] - offsets[r0]);
    }
    off += page_bytes;
  }
  if (page_off) page_off[npages] = off;
  return int64_t(off);
}

int64_t orc_encode_str(const uint8_t* bytes, const uint64_t* offsets, uint64_t n,
                       uint32_t page_rows, uint8_t* out, uint64_t cap, uint64_t* page_off,
                       uint64_t* row_prefix) {
  return encode_str_pages(STR, bytes, offsets, n, page_rows, out, cap, page_off, row_prefix);
}

// Decodes the string pages of a column (codec STR or FSST) back into byte
// offsets (n+1 entries, starting at 0) and the concatenated stored bytes.
static int64_t decode_str_pages(uint32_t codec, const uint8_t* blob, const uint64_t* page_off, uint64_t npages,
                                uint64_t n, uint32_t page_rows, uint64_t* offsets, uint8_t* bytes,
                                uint64_t bytes_cap) {
  uint64_t r = 0, pos = 0;
  offsets[0] = 0;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint8_t* pg = blob + page_off[p];
    uint32_t hdr[4];
    std::memcpy(hdr, pg, sizeof hdr);
    if (hdr[0] != (kMagic | (codec << 24))) return ECORRUPT;
    const uint32_t rows = hdr[1];
    if (rows == 0 || rows > page_rows || r + rows > n) return ECORRUPT;
    const uint32_t nmb = (rows + kMiniBlock - 1) / kMiniBlock;
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + hdr[2]);
    const uint8_t* region = pg + hdr[3];
    const uint64_t region_bytes = page_off[p + 1] - page_off[p] - hdr[3];
    for (uint32_t m = 0; m < nmb; ++m) {
      int32_t base;
      uint32_t wob, start;
      std::memcpy(&base, pg + kPageHeaderBytes + uint64_t(m) * 8, 4);
      std::memcpy(&wob, pg + kPageHeaderBytes + uint64_t(m) * 8 + 4, 4);
      std::memcpy(&start, pg + kPageHeaderBytes + uint64_t(nmb) * 8 + uint64_t(m) * 4, 4);
      const uint32_t bw = wob & 0xffu, woff = wob >> 8;
      if (bw > 32) return ECORRUPT;
      const uint32_t cnt = std::min<uint32_t>(kMiniBlock, rows - m * kMiniBlock);
      uint64_t s = start;
      for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t len = uint32_t(base) + unpack_bits(pay + woff, bw, j);
        if (s + len > region_bytes || pos + len > bytes_cap) return ECORRUPT;
        std::memcpy(bytes + pos, region + s, len);
        s += len;
        pos += len;
        offsets[r + j + 1] = pos;
      }
      r += cnt;
    }
  }
  return r == n ? OK : ECORRUPT;
}

int64_t orc_decode_str(const uint8_t* blob, const uint64_t* page_off, uint64_t npages, uint64_t n,
                       uint32_t page_rows, uint64_t* offsets, uint8_t* bytes, uint64_t bytes_cap) {
  return decode_str_pages(STR, blob, page_off, npages, n, page_rows, offsets, bytes, bytes_cap);
}

// ---------------------------------------------------------------------------
// FSST strings: the paper's string codec (Sec. 3.4.2, Sec. 4.1), written from
// the published method of Boncz, Neumann and Leis (FSST, VLDB 2020).  A
// symbol table holds up to 255 symbols of 1..8 bytes; an encoded string is a
// sequence of codes, code c < nsym standing for symbol c and code 255
// (escape) for the byte that follows it.  The table is kept with the column
// as nsym int32 triples {bytes 0..3, bytes 4..7 (little endian), length}.
// Pages: the STR page layout (codec FSST) over the encoded strings, whose
// lengths are the encoded lengths.
// ---------------------------------------------------------------------------
}  // extern "C"

constexpr uint32_t kFsstEscape = 255;
constexpr uint32_t kFsstMaxSymbols = 255;

// A symbol or an escaped byte: 1..8 bytes.
struct Tok {
  uint8_t len = 0;
  uint8_t b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool operator<(const Tok& o) const {
    const int c = std::memcmp(b, o.b, std::min(len, o.len));
    return c != 0 ? c < 0 : len < o.len;
  }
};

static Tok make_tok(const uint8_t* p, uint32_t len) {
  Tok t;
  t.len = uint8_t(len);
  std::memcpy(t.b, p, len);
  return t;
}

struct FsstSymbols {
  std::vector<Tok> sym;          // code -> bytes
  std::map<Tok, int> code;       // bytes -> code
};

static bool fsst_from_triples(const int32_t* t, uint64_t nt, FsstSymbols* out) {
  if (nt % 3 != 0 || nt / 3 > kFsstMaxSymbols) return false;
  out->sym.clear();
  out->code.clear();
  for (uint64_t i = 0; i < nt / 3; ++i) {
    const uint32_t len = uint32_t(t[3 * i + 2]);
    if (len < 1 || len > 8) return false;
    uint8_t b[8];
    std::memcpy(b, &t[3 * i], 4);
    std::memcpy(b + 4, &t[3 * i + 1], 4);
    const Tok s = make_tok(b, len);
    out->code.emplace(s, int(i));
    out->sym.push_back(s);
  }
  return true;
}

// Parses one string greedily with the table: at each position the longest
// symbol that matches, else an escaped byte.  Calls emit(token, code or -1).
template <class F>
static void fsst_parse(const FsstSymbols& T, const uint8_t* s, uint64_t len, F&& emit) {
  uint64_t i = 0;
  while (i < len) {
    int found = -1;
    uint32_t flen = 0;
    for (uint32_t L = uint32_t(std::min<uint64_t>(8, len - i)); L >= 1 && found < 0; --L) {
      auto it = T.code.find(make_tok(s + i, L));
      if (it != T.code.end()) {
        found = it->second;
        flen = L;
      }
    }
    if (found >= 0) {
      emit(make_tok(s + i, flen), found);
      i += flen;
    } else {
      emit(make_tok(s + i, 1), -1);
      i += 1;
    }
  }
}

extern "C" {

// Builds a symbol table from (a sample of) the strings, as the published
// method does: over a few generations, parse the sample with the current
// table, count how often each token (symbol or escaped byte) and each pair of
// consecutive tokens (when together at most 8 bytes) occurs, and keep the 255
// candidates of largest gain = count x length (ties: shorter, then smaller
// bytes).  Writes nsym triples to table (capacity 3 * 255); returns nsym.
int64_t orc_fsst_build(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, int32_t* table) {
  FsstSymbols T;
  const uint64_t sample = std::min<uint64_t>(n, 4096);
  for (int gen = 0; gen < 5; ++gen) {
    std::map<Tok, uint64_t> count;
    for (uint64_t r = 0; r < sample; ++r) {
      Tok prev;
      bool have_prev = false;
      fsst_parse(T, bytes + offsets[r], offsets[r + 1] - offsets[r], [&](const Tok& tok, int) {
        count[tok] += 1;
        if (have_prev && prev.len + tok.len <= 8) {
          Tok pair = prev;
          std::memcpy(pair.b + prev.len, tok.b, tok.len);
          pair.len = uint8_t(prev.len + tok.len);
          count[pair] += 1;
        }
        prev = tok;
        have_prev = true;
      });
    }
    std::vector<std::pair<Tok, uint64_t>> cand(count.begin(), count.end());
    std::sort(cand.begin(), cand.end(), [](const std::pair<Tok, uint64_t>& a, const std::pair<Tok, uint64_t>& b) {
      const uint64_t ga = a.second * a.first.len, gb = b.second * b.first.len;
      if (ga != gb) return ga > gb;
      if (a.first.len != b.first.len) return a.first.len < b.first.len;
      return a.first < b.first;
    });
    FsstSymbols next;
    for (size_t i = 0; i < cand.size() && next.sym.size() < kFsstMaxSymbols; ++i) {
      next.code.emplace(cand[i].first, int(next.sym.size()));
      next.sym.push_back(cand[i].first);
    }
    T = std::move(next);
  }
  for (size_t i = 0; i < T.sym.size(); ++i) {
    std::memcpy(&table[3 * i], T.sym[i].b, 4);
    std::memcpy(&table[3 * i + 1], T.sym[i].b + 4, 4);
    table[3 * i + 2] = int32_t(T.sym[i].len);
  }
  return int64_t(T.sym.size());
}

// Encodes the strings with the table and writes FSST pages (sizes as for
// orc_encode_str; out == NULL: sizes only).
int64_t orc_encode_fsst(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, const int32_t* table,
                        uint64_t ntab, uint32_t page_rows, uint8_t* out, uint64_t cap, uint64_t* page_off,
                        uint64_t* row_prefix) {
  FsstSymbols T;
  if (!fsst_from_triples(table, ntab, &T)) return EINVAL;
  std::vector<uint8_t> enc;
  std::vector<uint64_t> eoff(n + 1, 0);
  for (uint64_t r = 0; r < n; ++r) {
    fsst_parse(T, bytes + offsets[r], offsets[r + 1] - offsets[r], [&](const Tok& tok, int code) {
      if (code >= 0) {
        enc.push_back(uint8_t(code));
      } else {
        enc.push_back(uint8_t(kFsstEscape));
        enc.push_back(tok.b[0]);
      }
    });
    eoff[r + 1] = enc.size();
  }
  if (enc.empty()) enc.push_back(0);  // a valid pointer; no string reads it
  return encode_str_pages(FSST, enc.data(), eoff.data(), n, page_rows, out, cap, page_off, row_prefix);
}

// Decodes FSST pages back into the strings' byte offsets (n+1) and bytes.
int64_t orc_decode_fsst(const uint8_t* blob, const uint64_t* page_off, uint64_t npages, uint64_t n,
                        uint32_t page_rows, const int32_t* table, uint64_t ntab, uint64_t* offsets,
                        uint8_t* bytes, uint64_t bytes_cap) {
  FsstSymbols T;
  if (!fsst_from_triples(table, ntab, &T)) return EINVAL;
  const uint64_t stored_cap = page_off[npages];
  std::vector<uint64_t> eoff(n + 1);
  std::vector<uint8_t> enc(std::max<uint64_t>(stored_cap, 1));
  const int64_t st = decode_str_pages(FSST, blob, page_off, npages, n, page_rows, eoff.data(), enc.data(),
                                      enc.size());
  if (st < 0) return st;
  uint64_t pos = 0;
  offsets[0] = 0;
  for (uint64_t r = 0; r < n; ++r) {
    for (uint64_t i = eoff[r]; i < eoff[r + 1];) {
      const uint32_t c = enc[i++];
      if (c == kFsstEscape) {
        if (i >= eoff[r + 1] || pos + 1 > bytes_cap) return ECORRUPT;
        bytes[pos++] = enc[i++];
      } else {
        if (c >= T.sym.size()) return ECORRUPT;
        const Tok& sy = T.sym[c];
        if (pos + sy.len > bytes_cap) return ECORRUPT;
        std::memcpy(bytes + pos, sy.b, sy.len);
        pos += sy.len;
      }
    }
    offsets[r + 1] = pos;
  }
  return OK;
}

// ---------------------------------------------------------------------------
// Query evaluation over decoded columns.
// ---------------------------------------------------------------------------

enum PredOp : int32_t { LT = 0, LE, GT, GE, EQ, NE, BETWEEN, IN, PREFIX, CONTAINS, LIKE };
enum AggOp : int32_t { COUNT = 0, SUM, SUM_MUL, SUM_SUB };

struct OrcColumn {          // one decoded column
  int32_t is_str;
  const int32_t* v;         // 32-bit int columns (null for a 64-bit column)
  const uint8_t* bytes;     // string columns
  const uint64_t* offsets;  // n+1 byte offsets
  const int64_t* v64;       // 64-bit int columns (null otherwise)
};

// Integer value of row r (predicates and aggregates read 32-bit and 64-bit
// columns alike, as int64).
static int64_t ival(const OrcColumn& c, uint64_t r) { return c.v64 ? c.v64[r] : int64_t(c.v[r]); }

struct OrcTable {
  uint64_t n;
  int32_t ncols;
  const OrcColumn* cols;
};

// Joins, keys and payloads take 32-bit integer columns only.
static bool is_i32(const OrcTable& t, int32_t col) {
  return col >= 0 && col < t.ncols && !t.cols[col].is_str && t.cols[col].v != nullptr;
}

struct OrcPred {
  int32_t col, op, nargs, pfx_len;
  int64_t args[16];
  const uint8_t* pfx;
};

struct OrcJoin {
  int32_t fk_col;                 // column of the probing table (the fact, or the
                                  // dimension of the enclosing join)
  const OrcTable* dim;
  int32_t key_col;                // column of dim
  int32_t npreds;
  const OrcPred* preds;           // on dim
  int32_t npay;
  int32_t pay_cols[2];            // payload f: column pay_cols[f] of dim when
  int32_t pay_join[2];            //   pay_join[f] < 0, else field pay_field[f] of
  int32_t pay_field[2];           //   the row's match in sub join pay_join[f]
  int32_t nsub;                   // joins probed by dim's own scan (a chain:
  const struct OrcJoin* sub;      //   scan, probe, build of Sec. 3.1 Kernel #2)
};

struct OrcKey {
  int32_t kind;                   // 0: fact column, 1: join payload
  int32_t col, join, field;
};

struct OrcAgg {
  int32_t op, a, b;
};

struct OrcRecord {
  int32_t key[2];
  int64_t count;
  int64_t val[4];
};

// SQL LIKE over bytes, the whole string against the whole pattern: '%'
// stands for any run of bytes (possibly empty), '_' for any one byte, every
// other byte for itself (no escape character).  The textbook dynamic
// program: m[i][j] = the first i string bytes match the first j pattern
// bytes.
static bool like_match(const uint8_t* s, uint64_t n, const uint8_t* p, uint64_t k) {
  std::vector<std::vector<char>> m(n + 1, std::vector<char>(k + 1, 0));
  m[0][0] = 1;
  for (uint64_t j = 1; j <= k; ++j) m[0][j] = p[j - 1] == '%' && m[0][j - 1];
  for (uint64_t i = 1; i <= n; ++i)
    for (uint64_t j = 1; j <= k; ++j) {
      if (p[j - 1] == '%') m[i][j] = m[i][j - 1] || m[i - 1][j];             // empty run, or one more byte
      else m[i][j] = m[i - 1][j - 1] && (p[j - 1] == '_' || p[j - 1] == s[i - 1]);
    }
  return m[n][k] != 0;
}

static bool eval_pred(const OrcTable& t, const OrcPred& p, uint64_t r) {
  const OrcColumn& c = t.cols[p.col];
  if (p.op == LIKE) {
    const uint64_t len = c.offsets[r + 1] - c.offsets[r];
    return like_match(c.bytes + c.offsets[r], len, p.pfx, uint64_t(p.pfx_len));
  }
  if (p.op == PREFIX) {
    const uint64_t len = c.offsets[r + 1] - c.offsets[r];
    if (len < uint64_t(p.pfx_len)) return false;
    return std::memcmp(c.bytes + c.offsets[r], p.pfx, size_t(p.pfx_len)) == 0;
  }
  if (p.op == CONTAINS) {  // LIKE '%pattern%': the pattern occurs at some position
    const uint64_t len = c.offsets[r + 1] - c.offsets[r], m = uint64_t(p.pfx_len);
    if (m == 0) return true;
    for (uint64_t i = 0; i + m <= len; ++i)
      if (std::memcmp(c.bytes + c.offsets[r] + i, p.pfx, m) == 0) return true;
    return false;
  }
  const int64_t x = ival(c, r);
  switch (p.op) {
    case LT: return x < p.args[0];
    case LE: return x <= p.args[0];
    case GT: return x > p.args[0];
    case GE: return x >= p.args[0];
    case EQ: return x == p.args[0];
    case NE: return x != p.args[0];
    case BETWEEN: return p.args[0] <= x && x <= p.args[1];
    case IN:
      for (int32_t i = 0; i < p.nargs; ++i)
        if (x == p.args[i]) return true;
      return false;
  }
  return false;
}

using OrcMap = std::unordered_map<int32_t, std::vector<int32_t>>;

// The build side of one join: every row of J.dim that passes J's predicates
// and finds a match in each of J's sub joins (an inner join: a miss drops
// the row) maps its key to its payload values.  Sub joins are built first,
// the same way (Sec. 3.1: Kernel #1 scans and builds, Kernel #2 scans,
// probes the earlier table and builds the next).  Returns 0 or a status.
static int64_t build_map(const OrcJoin& J, OrcMap& m, int depth) {
  if (depth > 4 || J.nsub < 0 || J.nsub > 4 || J.npay < 0 || J.npay > 2) return EINVAL;
  if (!is_i32(*J.dim, J.key_col)) return EINVAL;
  for (int32_t s = 0; s < J.nsub; ++s)
    if (!is_i32(*J.dim, J.sub[s].fk_col)) return EINVAL;
  for (int32_t f = 0; f < J.npay; ++f)
    if (J.pay_join[f] < 0 && !is_i32(*J.dim, J.pay_cols[f])) return EINVAL;
  std::vector<OrcMap> subs(size_t(J.nsub));
  for (int32_t s = 0; s < J.nsub; ++s) {
    const int64_t rc = build_map(J.sub[s], subs[size_t(s)], depth + 1);
    if (rc) return rc;
  }
  for (int32_t f = 0; f < J.npay; ++f)
    if (J.pay_join[f] >= J.nsub || (J.pay_join[f] >= 0 && (J.pay_field[f] < 0 ||
                                                           J.pay_field[f] >= J.sub[J.pay_join[f]].npay)))
      return EINVAL;
  for (uint64_t r = 0; r < J.dim->n; ++r) {
    bool ok = true;
    for (int32_t k = 0; k < J.npreds && ok; ++k) ok = eval_pred(*J.dim, J.preds[k], r);
    std::vector<const std::vector<int32_t>*> hit(size_t(J.nsub), nullptr);
    for (int32_t s = 0; s < J.nsub && ok; ++s) {
      auto it = subs[size_t(s)].find(J.dim->cols[J.sub[s].fk_col].v[r]);
      if (it == subs[size_t(s)].end()) ok = false; else hit[size_t(s)] = &it->second;
    }
    if (!ok) continue;
    std::vector<int32_t> pay;
    for (int32_t f = 0; f < J.npay; ++f)
      pay.push_back(J.pay_join[f] < 0 ? J.dim->cols[J.pay_cols[f]].v[r]
                                      : (*hit[size_t(J.pay_join[f])])[size_t(J.pay_field[f])]);
    const int32_t key = J.dim->cols[J.key_col].v[r];
    if (!m.emplace(key, pay).second) return EDUPKEY;
  }
  return 0;
}

using OrcGroups = std::map<std::pair<int32_t, int32_t>, OrcRecord>;

// Checks the plan's shape and builds the join maps (the build side: key ->
// payload values of the dimension rows that pass).  Returns 0 or a status.
static int64_t prepare_query(const OrcTable* fact, int32_t njoins, const OrcJoin* joins, int32_t nkeys,
                             const OrcKey* keys, int32_t naggs, std::vector<OrcMap>& maps) {
  if (njoins < 0 || njoins > 8 || nkeys < 0 || nkeys > 2 || naggs < 0 || naggs > 4) return EINVAL;
  for (int32_t j = 0; j < njoins; ++j)
    if (!is_i32(*fact, joins[j].fk_col)) return EINVAL;
  for (int32_t k = 0; k < nkeys; ++k)
    if (keys[k].kind == 0 && !is_i32(*fact, keys[k].col)) return EINVAL;
  maps.assign(size_t(njoins), OrcMap());
  for (int32_t j = 0; j < njoins; ++j) {
    const int64_t rc = build_map(joins[j], maps[size_t(j)], 0);
    if (rc) return rc;
  }
  return 0;
}

// The probe side, one fact row at a time, over rows [r0, r1): predicates,
// then each join's lookup (a miss drops the row), then the row's group
// record, whose count and aggregates grow by this row's contribution.
static void eval_rows(const OrcTable* fact, uint64_t r0, uint64_t r1, int32_t npreds, const OrcPred* preds,
                      int32_t njoins, const OrcJoin* joins, const std::vector<OrcMap>& maps, int32_t nkeys,
                      const OrcKey* keys, int32_t naggs, const OrcAgg* aggs, OrcGroups& groups) {
  for (uint64_t r = r0; r < r1; ++r) {
    bool ok = true;
    for (int32_t k = 0; k < npreds && ok; ++k) ok = eval_pred(*fact, preds[k], r);
    if (!ok) continue;
    const std::vector<int32_t>* hit[8] = {};
    for (int32_t j = 0; j < njoins && ok; ++j) {
      auto it = maps[size_t(j)].find(fact->cols[joins[j].fk_col].v[r]);
      if (it == maps[size_t(j)].end()) ok = false; else hit[j] = &it->second;
    }
    if (!ok) continue;
    int32_t kv[2] = {0, 0};
    for (int32_t k = 0; k < nkeys; ++k)
      kv[k] = keys[k].kind == 0 ? fact->cols[keys[k].col].v[r] : (*hit[keys[k].join])[keys[k].field];
    auto ins = groups.emplace(std::make_pair(kv[0], kv[1]), OrcRecord{});
    OrcRecord& g = ins.first->second;
    if (ins.second) { g.key[0] = kv[0]; g.key[1] = kv[1]; }
    g.count += 1;
    for (int32_t a = 0; a < naggs; ++a) {
      const int64_t x = aggs[a].op == COUNT ? 0 : ival(fact->cols[aggs[a].a], r);
      const int64_t y = (aggs[a].op == SUM_MUL || aggs[a].op == SUM_SUB) ? ival(fact->cols[aggs[a].b], r) : 0;
      int64_t add = 0;
      switch (aggs[a].op) {   // int64 arithmetic modulo 2^64 (two's-complement wrap)
        case COUNT: add = 1; break;
        case SUM: add = x; break;
        case SUM_MUL: add = int64_t(uint64_t(x) * uint64_t(y)); break;
        case SUM_SUB: add = int64_t(uint64_t(x) - uint64_t(y)); break;
      }
      g.val[a] = int64_t(uint64_t(g.val[a]) + uint64_t(add));   // two's-complement wrap
    }
  }
}

// Writes the groups as records (ascending by key tuple; an ungrouped query
// always yields one record) and returns their number.
static int64_t emit_groups(OrcGroups& groups, int32_t nkeys, OrcRecord* out, uint64_t cap) {
  if (nkeys == 0 && groups.empty()) groups.emplace(std::make_pair(0, 0), OrcRecord{});
  uint64_t i = 0;
  for (const auto& kv : groups) {
    if (i < cap) out[i] = kv.second;
    ++i;
  }
  return int64_t(i);
}

// Evaluates the query.  Writes at most cap records (sorted ascending by key
// tuple, groups with zero rows omitted, an ungrouped query always yields one
// record) and returns the number of records, or a negative status.  This
// single-threaded walk over all fact rows is the definition.
int64_t orc_query(const OrcTable* fact, int32_t npreds, const OrcPred* preds, int32_t njoins,
                  const OrcJoin* joins, int32_t nkeys, const OrcKey* keys, int32_t naggs,
                  const OrcAgg* aggs, OrcRecord* out, uint64_t cap) {
  std::vector<OrcMap> maps;
  const int64_t rc = prepare_query(fact, njoins, joins, nkeys, keys, naggs, maps);
  if (rc) return rc;
  OrcGroups groups;
  eval_rows(fact, 0, fact->n, npreds, preds, njoins, joins, maps, nkeys, keys, naggs, aggs, groups);
  return emit_groups(groups, nkeys, out, cap);
}

// The same result from `nthreads` host threads: the fact rows are cut into
// ranges of `range_rows` rows (the page size, so a range is a run of whole
// pages), thread t evaluates ranges t, t + nthreads, ... into its own group
// map exactly as orc_query does, and the maps are merged by adding counts
// and aggregates modulo 2^64.  Integer addition is associative and
// commutative, so the merged records equal orc_query's.
int64_t orc_query_threads(const OrcTable* fact, int32_t npreds, const OrcPred* preds, int32_t njoins,
                          const OrcJoin* joins, int32_t nkeys, const OrcKey* keys, int32_t naggs,
                          const OrcAgg* aggs, OrcRecord* out, uint64_t cap, int32_t nthreads,
                          uint64_t range_rows) {
  if (nthreads < 1 || nthreads > 1024 || range_rows == 0) return EINVAL;
  std::vector<OrcMap> maps;
  const int64_t rc = prepare_query(fact, njoins, joins, nkeys, keys, naggs, maps);
  if (rc) return rc;
  const uint64_t nranges = (fact->n + range_rows - 1) / range_rows;
  std::vector<OrcGroups> part(static_cast<size_t>(nthreads));
  auto work = [&](int32_t t) {
    for (uint64_t i = uint64_t(t); i < nranges; i += uint64_t(nthreads)) {
      const uint64_t r0 = i * range_rows, r1 = std::min(fact->n, r0 + range_rows);
      eval_rows(fact, r0, r1, npreds, preds, njoins, joins, maps, nkeys, keys, naggs, aggs, part[size_t(t)]);
    }
  };
  std::vector<std::thread> pool;
  for (int32_t t = 1; t < nthreads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
  OrcGroups groups;
  for (const OrcGroups& p : part)
    for (const auto& kv : p) {
      auto ins = groups.emplace(kv.first, kv.second);
      if (ins.second) continue;
      OrcRecord& g = ins.first->second;
      g.count = int64_t(uint64_t(g.count) + uint64_t(kv.second.count));
      for (int a = 0; a < 4; ++a) g.val[a] = int64_t(uint64_t(g.val[a]) + uint64_t(kv.second.val[a]));
    }
  return emit_groups(groups, nkeys, out, cap);
}

}  // extern "C"

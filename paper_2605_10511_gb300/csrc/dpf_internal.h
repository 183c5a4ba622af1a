// Internal structures shared by the host side and the kernels of the library.
//
// The storage format (Sec. 3.4.1 fixed-length pages of mini blocks with a FOR
// base, a bit width and an offset; Sec. 3.4.2 variable-length pages and the
// RID index; Sec. 4.1 GPU-FOR; Sec. 4.2 page metadata) and the compiled
// device plan of one query pipeline (Sec. 3.1 Kernels #1-#3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dpf {

// ------------------------------------------------------------------ format
constexpr uint32_t kMB = 128;                 // values per mini block
constexpr uint32_t kPageHdr = 16;             // page header bytes
constexpr uint32_t kMagic = 0x00465044u;      // 'D' 'P' 'F', codec in the top byte
constexpr uint32_t kMaxPageRows = 1u << 20;
constexpr uint32_t kDefaultPageRows = 65536;

enum Codec : uint32_t { C_FOR = 1, C_DELTA = 2, C_DICT = 3, C_STR = 4, C_FSST = 5, C_FOR64 = 6 };
// STR and FSST share the variable-length page layout (FSST pages hold the
// encoded strings; their lengths are the encoded lengths).
__host__ __device__ inline bool is_str_codec(uint32_t codec) { return codec == C_STR || codec == C_FSST; }
constexpr uint32_t kFsstEscape = 255;     // FSST code: the next byte stands for itself
constexpr uint32_t kFsstMaxSymbols = 255;

// Bytes of one mini block header in the header array that follows the
// page header (STR: the lengths' FOR header; the u32 starts come after all
// headers).  FOR64 (Sec. 4.1, 64-bit GPU-FOR): {base: int64, word offset:
// u32 in 8-byte words, bit width: u32 in 0..64}; each mini block packs 128
// fields into 2 * bw 64-bit words.
__host__ __device__ inline uint32_t mb_hdr_bytes(uint32_t codec) {
  return codec == C_DELTA || codec == C_FOR64 ? 16u : 8u;
}
__host__ __device__ inline uint32_t mb_meta_bytes(uint32_t codec) {
  return codec == C_DELTA || codec == C_FOR64 ? 16u : (is_str_codec(codec) ? 12u : 8u);
}
__host__ __device__ inline uint64_t align16(uint64_t x) { return (x + 15u) & ~uint64_t(15); }
// Byte offset of the packed payload inside a page of `rows` rows.
__host__ __device__ inline uint32_t payload_offset(uint32_t codec, uint32_t rows) {
  const uint32_t nmb = (rows + kMB - 1) / kMB;
  return uint32_t(align16(kPageHdr + uint64_t(nmb) * mb_meta_bytes(codec)));
}

// ------------------------------------------------------------ device plan
constexpr int kMaxCols = 8;        // distinct fact columns one query touches
constexpr int kMaxSteps = 12;
constexpr int kMaxIn = 8;
constexpr int kMaxPrefix = 32;
constexpr int kMaxAggCols = 4;
constexpr int32_t kEmptyKey = int32_t(0x80000000);

// Device status bits (OR-ed into a status word, read by the host).
enum StatusBits : uint32_t { S_CORRUPT = 1u, S_INTERNAL = 2u, S_DUPKEY = 4u, S_TIMEOUT = 8u };

struct DevColumn {
  const uint8_t* blob;        // page images (device, or mapped pinned host)
  const uint64_t* page_off;   // [npages + 1] byte offset of each page (device)
  const int2* zone;           // [npages] bounds {lo, hi} of each page's values (device): a zone map
  const int4* sym;            // FSST: symbol table {bytes 0..3, bytes 4..7, length, 0} (device)
  uint64_t nrows;
  uint32_t codec;
  uint32_t page_rows;
  uint32_t max_bw;            // FOR/DICT/DELTA: widest mini block (bits), from the validated headers
  uint32_t nsym;              // FSST: symbols in the table
};

enum StepKind : uint8_t {
  ST_RANGE = 1,     // lo <= x <= hi
  ST_NOTRANGE = 2,  // !(lo <= x <= hi)
  ST_IN = 3,        // x in in[0..nin)
  ST_FALSE = 4,     // no row passes (e.g. an equality on a value absent from a dictionary)
  ST_CONTAINS = 9,  // the string contains pfx[0..plen) (LIKE '%pattern%'), matched by KMP
  ST_LIKE = 10,     // SQL LIKE of the whole string against pfx[0..plen) ('%', '_' wildcards)
  ST_PREFIX = 5,    // STR column starts with pfx[0..plen)
  ST_PROBE = 6,     // hash probe; a miss drops the row, a hit adds payload fields to gid
  ST_KEY = 7,       // DICT column code added to gid
  ST_RANGE64 = 11,     // FOR64 column: lo64 <= x <= hi64 (int64 bounds in in[0..3]); never a first step
  ST_NOTRANGE64 = 12,  // FOR64 column: !(lo64 <= x <= hi64)
  ST_ALL = 13,      // every row passes, nothing decoded: the first step of a scan whose filters are all 64-bit
};

// int64 bounds of an ST_RANGE64 / ST_NOTRANGE64 step, kept in the IN
// operand words: in[0..1] = lo64 (low word first), in[2..3] = hi64.
__host__ __device__ inline int64_t step_bound64(const int32_t* in, int i) {
  return int64_t((uint64_t(uint32_t(in[2 * i + 1])) << 32) | uint64_t(uint32_t(in[2 * i])));
}
__host__ __device__ inline bool is_step64(uint8_t kind) { return kind == 11 || kind == 12; }

// Join tables (Sec. 3.1 hash tables; representation chosen at build):
//  HT_OPEN   open addressing, slots {key, payload}, linear probing;
//  HT_DIRECT dense key range: entry[key - kmin] = payload or kAbsent;
//  HT_RANK   large, sparsely filled key range: a rank directory of 16-byte
//            words {presence bits of keys 0-31 and of keys 32-63 of 64
//            consecutive keys, present keys before the word, present keys
//            before its key 32}, followed by the payloads of the present
//            keys in key order (rank_entry).
// payload = code0 | code1 << 16 (dictionary codes of the payload columns).
enum HtKind : uint8_t { HT_OPEN = 0, HT_DIRECT = 1, HT_RANK = 2 };
constexpr uint32_t kAbsent = 0xffffffffu;

struct DevStep {
  uint8_t kind, col, nin, plen;
  int32_t lo, hi;
  int32_t in[kMaxIn];     // IN operands; ST_CONTAINS: in[0..1] = a pattern of <= 8 bytes
                          // packed for the sliding-window compare
  // ST_PROBE
  const void* ht;         // OPEN: uint2 slots; DIRECT: uint32 entries; RANK: directory + payloads (global)
  uint32_t ht_mask;       // OPEN: capacity - 1 (power of two)
  int32_t kmin;           // DIRECT / RANK: smallest key
  uint32_t krange;        // DIRECT / RANK: keys covered (kmin + [0, krange))
  uint8_t ht_kind;
  uint8_t smem_width;     // 0: probe global memory; OPEN: 8 (slots copied);
                          // DIRECT: 1/2/4-byte entries holding this join's
                          // group-id contribution (all ones = absent);
                          // PREFIX / CONTAINS on an FSST column: 1 = the
                          // step's code-level matcher tables sit at smem_off
  uint16_t pad_;
  uint32_t smem_off;      // byte offset of the copy in the CTA's table region
  uint32_t mul0, mul1;    // gid multipliers of payload fields 0 and 1 (0 = unused)
  // Values a row needs to pass (a superset: [zlo, zhi] empty when nothing
  // passes; the full int32 range when the step cannot prune): the range of a
  // predicate, the key range of a join table.  Mini blocks whose header
  // bounds miss it are skipped by the first step.
  int32_t zlo, zhi;
  // ST_KEY
  uint32_t key_mul;
  uint8_t pfx[kMaxPrefix];
  uint8_t kmp[kMaxPrefix];  // ST_CONTAINS: Knuth-Morris-Pratt failure function of pfx
};

struct alignas(16) DevQuery {
  DevColumn cols[kMaxCols];
  DevStep steps[kMaxSteps];
  uint32_t ncols, nsteps, smem_table_bytes;
  uint32_t pf_step;            // 1: while a segment's tiles run the first step, their mini
                               // blocks of step 1's column are prefetched into L2 (step 1
                               // then reads them per survivor); 0: no prefetch
  uint64_t nrows;
  uint32_t page_rows;
  uint32_t chunk_rows;
  uint64_t chunk_begin;        // first global ticket of this query
  uint64_t nchunks;
  // The launch's last tickets are cut smaller so that warps finish together:
  // tickets from tail_first on cover tail_rows rows each, starting at row
  // tail_first * chunk_rows (tail_rows == 0: every ticket covers chunk_rows).
  uint64_t tail_first;
  uint32_t tail_rows;
  uint32_t stage;              // > 0: the first step's mini blocks are staged in the warp's
                               // shared-memory ring, whose slots hold up to `stage` bits a value
  // aggregation: slot 0 = count, slot 1 + a = aggregate a
  uint32_t domain;             // number of dense group ids
  uint32_t naggs;
  uint8_t agg_op[4], agg_a[4], agg_b[4];   // agg_a/agg_b: column indices
  uint32_t use_smem_acc;
  uint32_t warp_agg;           // 1: warp-aggregated group-by updates (__match_any_sync peers)
  // group key reconstruction: code_k = (gid / key_div[k]) % key_dom[k]
  uint32_t nkeys;
  uint32_t key_div[2], key_dom[2];
  const int32_t* key_dict[2];
  // scratch and output (device)
  unsigned long long* acc;     // [domain][1 + naggs], zero between launches
  unsigned int* done;          // chunks flushed so far, zero between launches
  void* out;                   // dpf_record[domain]
  unsigned int* out_n;
  // dimension scans (hash build): key column and the sources of the payload
  // fields (a DICT column, a probed table's field, or group-id bits)
  int32_t build_key, build_npay, build_pay[2];
};

// A query needs the fused kernel's general string matcher when it has a
// CONTAINS or LIKE step or a string step on an FSST column.
inline bool needs_string_matcher(const DevQuery& Q) {
  for (uint32_t s = 0; s < Q.nsteps && s < uint32_t(kMaxSteps); ++s) {
    const DevStep& S = Q.steps[s];
    if (S.kind == ST_CONTAINS || S.kind == ST_LIKE || (S.kind == ST_PREFIX && Q.cols[S.col].codec == C_FSST))
      return true;
  }
  return false;
}

struct Sched {
  unsigned long long next;     // ticket counter
  unsigned int exited;         // CTAs that left the persistent loop
  unsigned int status;         // StatusBits
};

}  // namespace dpf

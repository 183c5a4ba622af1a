// Host side of the C ABI: context and memory accounting, column loading and
// page validation, the plan compiler (SQL-like plan -> device steps), hash
// builds and the prepared-batch launch / result path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dpf_internal.h"
#include "host_common.h"
#include "build_pay.h"
#include "kernels.h"

namespace dpf {

static thread_local std::string t_last_error;

dpf_status fail(dpf_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

unsigned host_threads() {
  const unsigned n = std::thread::hardware_concurrency();
  return std::max(1u, std::min(n == 0 ? 4u : n, 32u));
}

}  // namespace dpf

using namespace dpf;

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) return fail(DPF_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

struct Column {
  int32_t id = 0, codec = 0, placement = 0, table = 0;
  uint32_t page_rows = 0;
  uint64_t nrows = 0, npages = 0, bytes = 0, raw_bytes = 0;
  uint8_t* blob = nullptr;        // address the kernel reads (device or mapped host)
  uint8_t* host_blob = nullptr;   // pinned host allocation (HOST_PINNED)
  uint64_t* d_page_off = nullptr;
  int2* d_zone = nullptr;         // per-page value bounds (zone map)
  int4* d_sym = nullptr;          // FSST: symbol table {bytes 0..3, bytes 4..7, length, 0}
  int32_t* d_dict = nullptr;
  std::vector<uint64_t> page_off, row_prefix;
  std::vector<int32_t> dict;
  int64_t vmin = 0, vmax = -1;    // value bounds from the mini block headers (planner statistics)
  std::vector<int2> zones;        // host copy of the zone map (planner statistics)
  uint32_t max_bw = 0;            // FOR/DICT/DELTA: widest mini block (bits)
  uint64_t nsym = 0;              // FSST: symbols in the table
};

struct HashTable {
  int32_t id = 0, table = 0, npay = 0;
  int kind = HT_OPEN;
  uint2* slots = nullptr;         // HT_OPEN
  uint32_t capacity = 0;          // HT_OPEN slots, HT_DIRECT entries, HT_RANK keys covered
  uint32_t* direct = nullptr;     // HT_DIRECT
  uint8_t* rank = nullptr;        // HT_RANK: directory words, then payloads
  uint8_t* stage = nullptr;       // HT_RANK while building: pair count, then the staged pairs
  int32_t kmin = 0;
  uint64_t entries = 0;
  uint64_t dim_rows = 0;          // rows of the dimension the table was built from
  int32_t key_lo = 1, key_hi = 0; // smallest and largest stored key (empty: lo > hi)
  uint32_t pay_dom[2] = {0, 0};
  const int32_t* pay_dict[2] = {nullptr, nullptr};
  // asynchronous builds (dpf_build_hash_async) until finish_build
  bool pending = false;
  cudaEvent_t done = nullptr;     // recorded after the build's last kernel
  DevQuery* bq = nullptr;         // the build's compiled scan
  BuildStat* bstat = nullptr;     // its status word and inserted-row count
  dpf_col_id key_col = 0;
  dpf_status failed = DPF_OK;     // the error a finished build reported
  // tables sized before their scan keep their launch (dpf_build_hash_deferred:
  // rebuilt by every launch of the prepared chains that name them)
  bool deferred = false;
  int32_t refs = 0;               // prepared chains that rebuild the table
  BuildLaunch bl{};
  BuildStat* hstat = nullptr;     // deferred: pinned host copy of bstat, written by each chain launch
};

struct Prep {
  int32_t id = 0;
  int nq = 0;
  std::vector<DevQuery> hq;
  DevQuery* dq = nullptr;
  uint64_t* dqbegin = nullptr;
  Sched* sched = nullptr;
  uint8_t* scratch = nullptr;     // accumulators, counters, outputs of all queries
  FusedLaunch L{};
  dpf_tuning tuning{};
  cudaEvent_t ev = nullptr;
  bool launched = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool oneshot = false;
  std::vector<char> fetched;
  // unfused baseline chain
  bool unfused = false;
  UnfusedChain U{};
  uint8_t* unf_scratch = nullptr;
  uint32_t launches = 1;
  uint64_t fixed_inter_bytes = 0;   // decoded columns + flags per run
  // a prepared chain: these deferred tables are rebuilt, in order, before the
  // fused kernel of every launch (dpf_prepare_chain)
  std::vector<HashTable*> chain;
};

struct dpf_ctx {
  int device = 0;
  uint64_t budget = 0, used = 0;
  dpf_alloc_hooks hooks{};
  bool has_hooks = false;
  std::recursive_mutex mu;
  std::map<void*, uint64_t> dev_sizes;
  std::map<int32_t, Column> cols;
  std::map<int32_t, HashTable> hts;
  std::map<int32_t, std::unique_ptr<Prep>> preps;
  int32_t next_col = 1, next_ht = 1, next_prep = 1;
  cudaStream_t io = nullptr;      // private non-blocking stream for copies
  Sched* bsched = nullptr;        // status word of hash builds
  unsigned long long* bcount = nullptr;
  int32_t* bkminmax = nullptr;
  int num_sms = 0;
  int smem_optin = 0;
  std::map<uint64_t, dpf_tuning> tune_cache;  // plan-set signature -> tuning chosen by dpf_autotune
  dpf_tuning defaults{};          // dpf_set_tuning: fields a prepare and the autotuner leave open
  // Freed device blocks kept for reuse (without allocation hooks): a batch's
  // scratch is allocated at dpf_prepare and freed at dpf_release, and
  // cudaFree would wait for every kernel on the device, serialising a
  // serving loop's overlapping batches.
  std::multimap<uint64_t, void*> cache;
  uint64_t cached = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr uint64_t kCacheMaxBytes = uint64_t(8) << 30;  // freed bytes kept for reuse
constexpr uint64_t kCacheMaxBlock = uint64_t(1) << 30;  // larger blocks are returned at once

void drop_cache(dpf_ctx* c) {
  for (auto& kv : c->cache) cudaFree(kv.second);
  c->cache.clear();
  c->cached = 0;
}

dpf_status dev_alloc(dpf_ctx* c, uint64_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~uint64_t(255);
  void* p = nullptr;
  if (!c->has_hooks) {
    // reuse a cached block of at most 25 % more than asked for
    auto it = c->cache.lower_bound(bytes);
    if (it != c->cache.end() && it->first <= bytes + bytes / 4) {
      bytes = it->first;
      p = it->second;
      c->cache.erase(it);
      c->cached -= bytes;
    } else if (c->budget && c->used + c->cached + bytes > c->budget) {
      drop_cache(c);
    }
  }
  if (c->budget && c->used + bytes > c->budget) {
    if (p) {
      c->cache.emplace(bytes, p);
      c->cached += bytes;
    }
    return fail(DPF_ENOMEM, "device budget exceeded: %llu used + %llu > %llu", (unsigned long long)c->used,
                (unsigned long long)bytes, (unsigned long long)c->budget);
  }
  if (!p) {
    if (c->has_hooks) {
      p = c->hooks.alloc(bytes, c->hooks.user);
      if (!p) return fail(DPF_ENOMEM, "allocation hook failed for %llu bytes", (unsigned long long)bytes);
    } else {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess && !c->cache.empty()) {  // give the cached blocks back and retry
        cudaGetLastError();
        drop_cache(c);
        e = cudaMalloc(&p, bytes);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DPF_ENOMEM, "cudaMalloc(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
      }
    }
  }
  c->dev_sizes[p] = bytes;
  c->used += bytes;
  *out = p;
  return DPF_OK;
}

void dev_free(dpf_ctx* c, void* p) {
  if (!p) return;
  auto it = c->dev_sizes.find(p);
  if (it == c->dev_sizes.end()) return;
  const uint64_t bytes = it->second;
  c->used -= bytes;
  c->dev_sizes.erase(it);
  if (c->has_hooks) {
    c->hooks.free(p, c->hooks.user);
  } else if (bytes <= kCacheMaxBlock && c->cached + bytes <= kCacheMaxBytes &&
             (!c->budget || c->used + c->cached + bytes <= c->budget)) {
    c->cache.emplace(bytes, p);
    c->cached += bytes;
  } else {
    cudaFree(p);
  }
}

// Frees a table's device blocks (and an asynchronous build's launch buffers).
static void free_table(dpf_ctx* c, HashTable& ht) {
  dev_free(c, ht.slots);
  dev_free(c, ht.direct);
  dev_free(c, ht.rank);
  dev_free(c, ht.stage);
  dev_free(c, ht.bq);
  dev_free(c, ht.bstat);
  if (ht.hstat) cudaFreeHost(ht.hstat);
  if (ht.done) cudaEventDestroy(ht.done);
  ht.slots = nullptr;
  ht.direct = nullptr;
  ht.rank = nullptr;
  ht.stage = nullptr;
  ht.bq = nullptr;
  ht.bstat = nullptr;
  ht.hstat = nullptr;
  ht.done = nullptr;
}

// Enqueues the build of a table sized before its scan on s: its status
// zeroed, the table emptied (absent entries, no presence bits, no staged
// pairs), the insert pass(es), then the event dpf_hash_wait waits on.
static cudaError_t enqueue_table_build(HashTable& ht, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ht.bstat, 0, sizeof(BuildStat), s);
  if (e == cudaSuccess) {
    if (ht.kind == HT_RANK) {
      e = cudaMemsetAsync(ht.rank, 0, 16 * ((uint64_t(ht.capacity) + 63) / 64), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(ht.stage, 0, 16, s);
    } else if (ht.kind == HT_DIRECT) {
      e = launch_init_direct(ht.direct, std::max<uint32_t>(ht.capacity, 1u), s);
    } else {
      e = launch_init_table(ht.slots, ht.capacity, s);
    }
  }
  if (e == cudaSuccess) e = launch_build_insert(ht.bl, s);
  if (e == cudaSuccess && ht.hstat) e = cudaMemcpyAsync(ht.hstat, ht.bstat, sizeof(BuildStat), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) {
    // captured into a graph, the record must be an external event node for
    // the host to wait on it after a replay
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e == cudaSuccess)
      e = cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ht.done, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ht.done, s);
  }
  return e;
}

template <class T>
dpf_status dev_alloc_t(dpf_ctx* c, uint64_t count, T** out) {
  void* p;
  dpf_status st = dev_alloc(c, count * sizeof(T), &p);
  *out = static_cast<T*>(p);
  return st;
}

dpf_status upload(dpf_ctx* c, void* dst, const void* src, uint64_t bytes) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->io));
  CUDA_TRY(cudaStreamSynchronize(c->io));
  return DPF_OK;
}

void free_column(dpf_ctx* c, Column& col) {
  if (col.placement == DPF_PLACE_HOST_PINNED) {
    if (col.host_blob) cudaFreeHost(col.host_blob);
  } else {
    dev_free(c, col.blob);
  }
  dev_free(c, col.d_page_off);
  dev_free(c, col.d_zone);
  dev_free(c, col.d_sym);
  dev_free(c, col.d_dict);
  col.blob = col.host_blob = nullptr;
}

// ---------------------------------------------------------------- validation
inline uint32_t rd32(const uint8_t* p) {
  uint32_t x;
  std::memcpy(&x, p, 4);
  return x;
}

// Checks every page and mini block header so that the kernels can trust
// offsets and widths (they still guard bit widths and group ids).
dpf_status validate_pages(uint32_t codec, const uint8_t* pages, uint64_t size, const uint64_t* page_off,
                          uint64_t npages, uint64_t nrows, uint32_t P, uint64_t dict_n) {
  if (page_off[0] != 0 || page_off[npages] != size) return fail(DPF_ECORRUPT, "page_off does not span the pages");
  bool bad = false;
  uint64_t bad_page = 0;
  std::mutex m;
  parallel_for(npages, [&](uint64_t p) {
    auto flag = [&] {
      std::lock_guard<std::mutex> g(m);
      if (!bad || p < bad_page) bad_page = p;
      bad = true;
    };
    const uint64_t a = page_off[p], b = page_off[p + 1];
    if (a % 16 || b < a || b - a < kPageHdr || b > size) return flag();
    const uint8_t* pg = pages + a;
    const uint64_t pbytes = b - a;
    const uint32_t rows = uint32_t(std::min<uint64_t>(P, nrows - p * uint64_t(P)));
    if (rd32(pg) != (kMagic | (codec << 24)) || rd32(pg + 4) != rows) return flag();
    const uint32_t poff = rd32(pg + 8), extra = rd32(pg + 12);
    if (poff != payload_offset(codec, rows) || poff > pbytes) return flag();
    const uint64_t pay_end = is_str_codec(codec) ? extra : pbytes;
    if (is_str_codec(codec) && (extra < poff || extra > pbytes || extra % 16)) return flag();
    const uint64_t pay_words = (pay_end - poff) / 4;
    const uint32_t nmb = (rows + kMB - 1) / kMB;
    if (codec == C_FOR64) {  // {base: int64, word offset: u32, bit width: u32}, 8-byte words
      for (uint32_t m2 = 0; m2 < nmb; ++m2) {
        const uint8_t* h = pg + kPageHdr + uint64_t(m2) * 16;
        const uint32_t woff = rd32(h + 8), bw = rd32(h + 12);
        if (bw > 64 || uint64_t(woff) + 2ull * bw > pay_words / 2) return flag();
      }
      return;
    }
    for (uint32_t m2 = 0; m2 < nmb; ++m2) {
      const uint8_t* h = pg + kPageHdr + uint64_t(m2) * mb_hdr_bytes(codec);
      const uint32_t wob = codec == C_DELTA ? rd32(h + 8) : rd32(h + 4);
      const uint32_t bw = wob & 0xffu, woff = wob >> 8;
      // a mini block's 4 * bw words start on a 16-byte boundary (the kernels
      // copy them in 16-byte chunks)
      if (bw > 32 || woff % 4 != 0 || uint64_t(woff) + 4ull * bw > pay_words) return flag();
      if (codec == C_DICT) {
        const int32_t base = int32_t(rd32(h));
        if (base < 0 || uint64_t(base) >= dict_n) return flag();
      }
      if (is_str_codec(codec)) {
        // lengths of the mini block must stay inside the page's byte region
        const uint32_t start = rd32(pg + kPageHdr + uint64_t(nmb) * 8 + uint64_t(m2) * 4);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(pg + poff) + woff;
        const uint32_t base = rd32(h);
        const uint32_t cnt = std::min<uint32_t>(kMB, rows - m2 * kMB);
        uint64_t sum = 0;
        for (uint32_t j = 0; j < cnt; ++j) {
          uint32_t f = 0;
          if (bw) {
            const uint64_t bit = uint64_t(j) * bw;
            uint64_t win = w[bit >> 5];
            if ((bit & 31) + bw > 32) win |= uint64_t(w[(bit >> 5) + 1]) << 32;
            f = uint32_t((win >> (bit & 31)) & (bw == 32 ? 0xffffffffull : ((1ull << bw) - 1)));
          }
          sum += uint64_t(base) + f;
        }
        if (uint64_t(start) + sum > pbytes - extra) return flag();
      }
    }
  });
  if (bad) return fail(DPF_ECORRUPT, "page %llu failed validation", (unsigned long long)bad_page);
  return DPF_OK;
}

// ---------------------------------------------------------------- plans
// Every FSST code of every string must name a symbol of the table, and an
// escape must be followed by its literal inside the same string, so the
// kernels can decode without bounds checks on the table.
dpf_status validate_fsst_codes(const uint8_t* pages, const uint64_t* page_off, uint64_t npages, uint64_t nrows,
                               uint32_t P, uint32_t nsym) {
  bool bad = false;
  std::mutex m;
  parallel_for(npages, [&](uint64_t p) {
    const uint8_t* pg = pages + page_off[p];
    const uint32_t rows = uint32_t(std::min<uint64_t>(P, nrows - p * uint64_t(P)));
    const uint32_t nmb = (rows + kMB - 1) / kMB;
    const uint8_t* region = pg + rd32(pg + 12);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(pg + rd32(pg + 8));
    for (uint32_t mb = 0; mb < nmb && !bad; ++mb) {
      const uint8_t* h = pg + kPageHdr + uint64_t(mb) * 8;
      const uint32_t base = rd32(h), wob = rd32(h + 4), bw = wob & 0xffu;
      uint64_t pos = rd32(pg + kPageHdr + uint64_t(nmb) * 8 + uint64_t(mb) * 4);
      const uint32_t cnt = std::min<uint32_t>(kMB, rows - mb * kMB);
      for (uint32_t j = 0; j < cnt; ++j) {
        uint32_t f = 0;
        if (bw) {
          const uint64_t bit = uint64_t(j) * bw;
          uint64_t win = pay[(wob >> 8) + (bit >> 5)];
          if ((bit & 31) + bw > 32) win |= uint64_t(pay[(wob >> 8) + (bit >> 5) + 1]) << 32;
          f = uint32_t((win >> (bit & 31)) & (bw == 32 ? 0xffffffffull : ((1ull << bw) - 1)));
        }
        const uint64_t end = pos + base + f;
        for (uint64_t i = pos; i < end;) {
          const uint32_t code = region[i++];
          if (code == kFsstEscape) {
            if (i >= end) { std::lock_guard<std::mutex> g(m); bad = true; break; }
            ++i;
          } else if (code >= nsym) {
            std::lock_guard<std::mutex> g(m);
            bad = true;
            break;
          }
        }
        pos = end;
      }
    }
  });
  return bad ? fail(DPF_ECORRUPT, "an FSST code names no symbol of the table, or an escape ends a string") : DPF_OK;
}

dpf_status compile_pred_body(const Column& c, const dpf_pred& p, DevStep& S, int col_index) {
  std::memset(&S, 0, sizeof S);
  S.col = uint8_t(col_index);
  if (c.codec == C_FOR64) {
    // BIGINT (Sec. 4.1, 64-bit GPU-FOR): the int64 value against int64
    // operands, as an int64 range or its complement
    int64_t lo = INT64_MIN, hi = INT64_MAX;
    bool neg = false;
    switch (p.op) {
      case DPF_OP_LT:
        if (p.v[0] == INT64_MIN) lo = 1, hi = 0;
        else hi = p.v[0] - 1;
        break;
      case DPF_OP_LE: hi = p.v[0]; break;
      case DPF_OP_GT:
        if (p.v[0] == INT64_MAX) lo = 1, hi = 0;
        else lo = p.v[0] + 1;
        break;
      case DPF_OP_GE: lo = p.v[0]; break;
      case DPF_OP_EQ: lo = hi = p.v[0]; break;
      case DPF_OP_NE: lo = hi = p.v[0]; neg = true; break;
      case DPF_OP_BETWEEN: lo = p.v[0]; hi = p.v[1]; break;
      case DPF_OP_IN:
        if (p.n != 1) return fail(DPF_EINVAL, "IN on FOR64 column %d takes one operand (got %d)", c.id, p.n);
        lo = hi = p.v[0];
        break;
      default: return fail(DPF_EINVAL, "predicate op %d does not apply to FOR64 column %d", p.op, c.id);
    }
    S.kind = neg ? ST_NOTRANGE64 : ST_RANGE64;
    S.in[0] = int32_t(uint32_t(uint64_t(lo)));
    S.in[1] = int32_t(uint32_t(uint64_t(lo) >> 32));
    S.in[2] = int32_t(uint32_t(uint64_t(hi)));
    S.in[3] = int32_t(uint32_t(uint64_t(hi) >> 32));
    return DPF_OK;
  }
  if (p.op == DPF_OP_PREFIX || p.op == DPF_OP_CONTAINS || p.op == DPF_OP_LIKE) {
    if (!is_str_codec(uint32_t(c.codec)))
      return fail(DPF_EINVAL, "PREFIX / CONTAINS / LIKE need a STR or FSST column (column %d)", c.id);
    if (p.prefix_len < 0 || p.prefix_len > DPF_MAX_PREFIX) return fail(DPF_EINVAL, "prefix_len %d out of range", p.prefix_len);
    int32_t op = p.op;
    const uint8_t* pat = p.prefix;
    int32_t plen = p.prefix_len;
    if (op == DPF_OP_LIKE) {
      // 'p%' is PREFIX p and '%p%' is CONTAINS p when p has no wildcard
      bool inner_wild = false;
      const bool lead = plen > 0 && pat[0] == '%', trail = plen > (lead ? 1 : 0) && pat[plen - 1] == '%';
      for (int32_t i = lead ? 1 : 0; i < plen - (trail ? 1 : 0); ++i) inner_wild |= pat[i] == '%' || pat[i] == '_';
      bool all_pct = plen > 0;
      for (int32_t i = 0; i < plen; ++i) all_pct = all_pct && pat[i] == '%';
      if (all_pct) {  // only '%': every string matches
        op = DPF_OP_CONTAINS;
        plen = 0;
      } else if (!inner_wild && trail) {
        op = lead ? DPF_OP_CONTAINS : DPF_OP_PREFIX;
        pat += lead ? 1 : 0;
        plen -= (lead ? 1 : 0) + 1;
      } else if (c.codec != C_STR) {
        return fail(DPF_EINVAL, "LIKE patterns other than 'p%%' and '%%p%%' need a STR column (column %d is FSST)",
                    c.id);
      }
    }
    S.kind = op == DPF_OP_PREFIX ? ST_PREFIX : op == DPF_OP_CONTAINS ? ST_CONTAINS : ST_LIKE;
    S.plen = uint8_t(plen);
    std::memcpy(S.pfx, pat, size_t(plen));
    if (S.kind == ST_CONTAINS) {
      // a pattern of <= 8 bytes packed for the sliding-window compare: byte k
      // of the pattern at bits 8 * (plen - 1 - k) (the newest byte lowest)
      uint64_t pat = 0;
      for (uint32_t k = 0; k < S.plen && S.plen <= 8; ++k) pat |= uint64_t(S.pfx[k]) << (8 * (S.plen - 1 - k));
      S.in[0] = int32_t(uint32_t(pat));
      S.in[1] = int32_t(uint32_t(pat >> 32));
      // Knuth-Morris-Pratt failure function: kmp[i] = length of the longest
      // proper border of pattern[0..i]
      uint32_t k = 0;
      if (S.plen) S.kmp[0] = 0;
      for (uint32_t i = 1; i < S.plen; ++i) {
        while (k > 0 && S.pfx[i] != S.pfx[k]) k = S.kmp[k - 1];
        if (S.pfx[i] == S.pfx[k]) ++k;
        S.kmp[i] = uint8_t(k);
      }
    }
    return DPF_OK;
  }
  if (is_str_codec(uint32_t(c.codec)))
    return fail(DPF_EINVAL, "only PREFIX, CONTAINS and LIKE apply to string column %d", c.id);
  const int64_t MN = INT32_MIN, MX = INT32_MAX;
  int64_t lo, hi;
  bool neg = false;
  switch (p.op) {
    case DPF_OP_LT: lo = MN; hi = p.v[0] - 1; break;
    case DPF_OP_LE: lo = MN; hi = p.v[0]; break;
    case DPF_OP_GT: lo = p.v[0] + 1; hi = MX; break;
    case DPF_OP_GE: lo = p.v[0]; hi = MX; break;
    case DPF_OP_EQ: lo = hi = p.v[0]; break;
    case DPF_OP_NE: lo = hi = p.v[0]; neg = true; break;
    case DPF_OP_BETWEEN: lo = p.v[0]; hi = p.v[1]; break;
    case DPF_OP_IN: {
      if (p.n < 1 || p.n > DPF_MAX_IN) return fail(DPF_EINVAL, "IN takes 1..%d operands", DPF_MAX_IN);
      std::vector<int32_t> vals;
      for (int i = 0; i < p.n; ++i) {
        const int64_t x = p.v[i];
        if (c.codec == C_DICT) {
          auto it = std::lower_bound(c.dict.begin(), c.dict.end(), x,
                                     [](int32_t a, int64_t b) { return int64_t(a) < b; });
          if (it != c.dict.end() && int64_t(*it) == x) vals.push_back(int32_t(it - c.dict.begin()));
        } else if (x >= MN && x <= MX) {
          vals.push_back(int32_t(x));
        }
      }
      if (vals.empty()) { S.kind = ST_FALSE; return DPF_OK; }
      S.kind = ST_IN;
      S.nin = uint8_t(vals.size());
      for (size_t i = 0; i < vals.size(); ++i) S.in[i] = vals[i];
      return DPF_OK;
    }
    default: return fail(DPF_EINVAL, "unknown predicate op %d", p.op);
  }
  if (c.codec == C_DICT) {
    // value interval -> code interval over the sorted dictionary
    auto lb = [&](int64_t x) {
      return int64_t(std::lower_bound(c.dict.begin(), c.dict.end(), x,
                                      [](int32_t a, int64_t b) { return int64_t(a) < b; }) - c.dict.begin());
    };
    const int64_t clo = lb(lo);
    const int64_t chi = hi == INT64_MAX ? int64_t(c.dict.size()) - 1 : lb(hi + 1) - 1;
    if (neg) {
      if (clo > chi) { S.kind = ST_RANGE; S.lo = INT32_MIN; S.hi = INT32_MAX; return DPF_OK; }
      S.kind = ST_NOTRANGE; S.lo = int32_t(clo); S.hi = int32_t(chi);
      return DPF_OK;
    }
    if (clo > chi) { S.kind = ST_FALSE; return DPF_OK; }
    S.kind = ST_RANGE; S.lo = int32_t(clo); S.hi = int32_t(chi);
    return DPF_OK;
  }
  lo = std::max(lo, MN);
  hi = std::min(hi, MX);
  if (neg) {
    if (lo > hi) { S.kind = ST_RANGE; S.lo = INT32_MIN; S.hi = INT32_MAX; return DPF_OK; }
    S.kind = ST_NOTRANGE; S.lo = int32_t(lo); S.hi = int32_t(hi);
    return DPF_OK;
  }
  if (lo > hi) { S.kind = ST_FALSE; return DPF_OK; }
  S.kind = ST_RANGE; S.lo = int32_t(lo); S.hi = int32_t(hi);
  return DPF_OK;
}

// Compiles one predicate and sets the value range a row needs to pass it
// (used to skip mini blocks whose header bounds miss it).
dpf_status compile_pred(const Column& c, const dpf_pred& p, DevStep& S, int col_index) {
  const dpf_status st = compile_pred_body(c, p, S, col_index);
  if (st) return st;
  S.zlo = INT32_MIN;
  S.zhi = INT32_MAX;
  if (S.kind == ST_RANGE) {
    S.zlo = S.lo;
    S.zhi = S.hi;
  } else if (S.kind == ST_IN) {
    S.zlo = *std::min_element(S.in, S.in + S.nin);
    S.zhi = *std::max_element(S.in, S.in + S.nin);
  } else if (S.kind == ST_FALSE) {
    S.zlo = 1;
    S.zhi = 0;
  }
  return DPF_OK;
}

// Value bounds of a column, read from its validated mini block headers: per
// page (a zone map the kernel uses to skip pages) and for the whole column
// (planner statistics).  FOR and DICT (codes): [base, base + 2^bw - 1] per
// mini block (the upper end is a bound, not exact).  DELTA: every value lies
// within 127 steps of the mini block's first value, each step in
// [min(0, dmin), max(0, dmin + 2^bw - 1)]; a page whose bound leaves int32
// (values may have wrapped) gets the full range.  STR: the full range.
void value_bounds(uint32_t codec, const uint8_t* pages, const uint64_t* page_off, uint64_t npages, uint64_t nrows,
                  uint32_t P, int64_t* vmin, int64_t* vmax, std::vector<int2>* zones, uint32_t* max_bw) {
  *vmin = 0;
  *vmax = -1;
  *max_bw = 0;
  zones->assign(npages, make_int2(INT32_MIN, INT32_MAX));
  if (is_str_codec(codec) || codec == C_FOR64) return;  // no 32-bit bounds (never a step's column)
  int64_t clo = INT64_MAX, chi = INT64_MIN;
  for (uint64_t p = 0; p < npages; ++p) {
    const uint8_t* pg = pages + page_off[p];
    const uint32_t rows = uint32_t(std::min<uint64_t>(P, nrows - p * uint64_t(P)));
    const uint32_t nmb = (rows + kMB - 1) / kMB;
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (uint32_t m = 0; m < nmb; ++m) {
      const uint8_t* h = pg + kPageHdr + uint64_t(m) * mb_hdr_bytes(codec);
      const int64_t base = int32_t(rd32(h));
      if (codec == C_DELTA) {
        const int64_t dmin = int32_t(rd32(h + 4));
        const uint32_t bw = std::min<uint32_t>(rd32(h + 8) & 0xffu, 32u);
        *max_bw = std::max(*max_bw, bw);
        const int64_t span = bw >= 32 ? int64_t(0xffffffffll) : (int64_t(1) << bw) - 1;
        lo = std::min(lo, base + 127 * std::min<int64_t>(0, dmin));
        hi = std::max(hi, base + 127 * std::max<int64_t>(0, dmin + span));
      } else {
        const uint32_t bw = std::min<uint32_t>(rd32(h + 4) & 0xffu, 32u);
        *max_bw = std::max(*max_bw, bw);
        lo = std::min(lo, base);
        hi = std::max(hi, base + (bw >= 32 ? int64_t(0xffffffffll) : (int64_t(1) << bw) - 1));
      }
    }
    if (lo > hi) continue;
    clo = std::min(clo, lo);
    chi = std::max(chi, hi);
    if (lo >= INT32_MIN && hi <= INT32_MAX) (*zones)[p] = make_int2(int32_t(lo), int32_t(hi));
  }
  if (clo <= chi) {
    *vmin = std::max<int64_t>(clo, INT32_MIN);
    *vmax = std::min<int64_t>(chi, INT32_MAX);
  }
}

// Fraction of a column's rows in pages whose zone map meets [lo, hi]: the
// rows a first step over that range decodes (the kernel skips the other
// pages unread).
double zone_fraction(const Column& col, int32_t lo, int32_t hi) {
  if (col.nrows == 0 || col.zones.empty()) return 1.0;
  if (lo > hi) return 0.0;
  uint64_t kept = 0;
  for (uint64_t p = 0; p < col.zones.size(); ++p) {
    const int2 z = col.zones[p];
    if (z.y < lo || z.x > hi) continue;
    kept += std::min<uint64_t>(col.page_rows, col.nrows - p * uint64_t(col.page_rows));
  }
  return double(kept) / double(col.nrows);
}

// Estimated fraction of rows a step keeps, for ordering the steps: range
// predicates assume values spread evenly over the column's bounds; a join
// keeps the fraction of dimension rows that passed its build predicates
// (foreign keys spread over the dimension); group keys keep every row.
double step_selectivity(const DevStep& S, const Column* col, const HashTable* ht) {
  switch (S.kind) {
    case ST_FALSE: return 0.0;
    case ST_KEY: return 2.0;  // not a filter: after every filter
    case ST_PROBE: return ht && ht->dim_rows ? double(ht->entries) / double(ht->dim_rows) : 1.0;
    case ST_RANGE64:
    case ST_NOTRANGE64: return 0.5;  // no 64-bit value bounds are kept
    case ST_ALL: return 1.0;
    case ST_PREFIX: return std::pow(0.1, double(S.plen));
    case ST_CONTAINS: return std::min(1.0, 30.0 * std::pow(0.1, double(S.plen)));
    case ST_LIKE: {
      double lits = 0;
      for (uint32_t i = 0; i < S.plen; ++i) lits += S.pfx[i] != '%' && S.pfx[i] != '_';
      return std::min(1.0, 30.0 * std::pow(0.1, lits));
    }
    default: break;
  }
  if (!col || col->vmax < col->vmin) return 0.5;
  const double width = double(col->vmax - col->vmin) + 1.0;
  if (S.kind == ST_IN) return std::min(1.0, double(S.nin) / width);
  const double lo = std::max<double>(double(S.lo), double(col->vmin));
  const double hi = std::min<double>(double(S.hi), double(col->vmax));
  const double in = hi >= lo ? (hi - lo + 1.0) / width : 0.0;
  return S.kind == ST_NOTRANGE ? 1.0 - in : in;
}

struct ColumnSet {
  dpf_ctx* c;
  DevQuery& Q;
  std::vector<int32_t> ids;
  int32_t table = -1;
  uint64_t nrows = 0;
  uint32_t page_rows = 0;
  bool host = false;
  // The table checks of add without adding the column (a column a plan
  // names but never reads).
  dpf_status check(int32_t id) const {
    auto it = c->cols.find(id);
    if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", id);
    const Column& col = it->second;
    if (!ids.empty() && (col.table != table || col.nrows != nrows || col.page_rows != page_rows))
      return fail(DPF_EINVAL, "column %d is not in the same table (table/rows/page_rows differ)", id);
    return DPF_OK;
  }
  dpf_status add(int32_t id, int* idx) {
    auto it = c->cols.find(id);
    if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", id);
    const Column& col = it->second;
    for (size_t i = 0; i < ids.size(); ++i)
      if (ids[i] == id) { *idx = int(i); return DPF_OK; }
    if (ids.empty()) {
      table = col.table; nrows = col.nrows; page_rows = col.page_rows;
    } else if (col.table != table || col.nrows != nrows || col.page_rows != page_rows) {
      return fail(DPF_EINVAL, "column %d is not in the same table (table/rows/page_rows differ)", id);
    }
    if (ids.size() >= size_t(kMaxCols)) return fail(DPF_EINVAL, "a plan may touch at most %d columns", kMaxCols);
    DevColumn& d = Q.cols[ids.size()];
    d.blob = col.blob;
    d.page_off = col.d_page_off;
    d.zone = col.d_zone;
    d.sym = col.d_sym;
    d.nrows = col.nrows;
    d.codec = uint32_t(col.codec);
    d.page_rows = col.page_rows;
    d.max_bw = col.max_bw;
    d.nsym = col.codec == C_FSST ? uint32_t(col.nsym) : 0u;
    host |= col.placement == DPF_PLACE_HOST_PINNED;
    *idx = int(ids.size());
    ids.push_back(id);
    Q.ncols = uint32_t(ids.size());
    return DPF_OK;
  }
};

dpf_status compile_plan(dpf_ctx* c, const dpf_plan& P, DevQuery& Q, bool* host,
                        std::vector<const HashTable*>& probes) {
  std::memset(&Q, 0, sizeof Q);
  ColumnSet cs{c, Q};
  if (P.n_preds < 0 || P.n_preds > DPF_MAX_PREDS || P.n_joins < 0 || P.n_joins > DPF_MAX_JOINS ||
      P.n_keys < 0 || P.n_keys > DPF_MAX_KEYS || P.n_aggs < 0 || P.n_aggs > DPF_MAX_AGGS)
    return fail(DPF_EINVAL, "plan sizes out of range");
  if ((P.n_preds && !P.preds) || (P.n_joins && !P.joins) || (P.n_keys && !P.keys) || (P.n_aggs && !P.aggs))
    return fail(DPF_EINVAL, "plan array pointer is NULL");
  std::vector<DevStep> steps;
  std::vector<double> sel;  // estimated selectivity of each step
  // A predicate every row passes (an empty PREFIX or CONTAINS pattern, LIKE
  // '%', a range over the whole int32 or int64 domain) compiles to no step:
  // its column is checked but not read.
  std::vector<int32_t> unread;
  for (int i = 0; i < P.n_preds; ++i) {
    if (c->cols.find(P.preds[i].col) == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", P.preds[i].col);
    DevStep S;
    dpf_status st = compile_pred(c->cols[P.preds[i].col], P.preds[i], S, 0);
    if (st) return st;
    const bool all = ((S.kind == ST_PREFIX || S.kind == ST_CONTAINS) && S.plen == 0) ||
                     (S.kind == ST_RANGE && S.lo == INT32_MIN && S.hi == INT32_MAX) ||
                     (S.kind == ST_RANGE64 && step_bound64(S.in, 0) == INT64_MIN && step_bound64(S.in, 1) == INT64_MAX) ||
                     (S.kind == ST_NOTRANGE64 && step_bound64(S.in, 0) > step_bound64(S.in, 1));
    if (all) {
      unread.push_back(P.preds[i].col);
      continue;
    }
    int idx;
    if ((st = cs.add(P.preds[i].col, &idx))) return st;
    S.col = uint8_t(idx);
    sel.push_back(step_selectivity(S, &c->cols[P.preds[i].col], nullptr));
    steps.push_back(S);
  }
  probes.clear();
  std::vector<size_t> probe_step;
  for (int j = 0; j < P.n_joins; ++j) {
    const dpf_join& J = P.joins[j];
    auto ht = c->hts.find(J.ht);
    if (ht == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", J.ht);
    if (ht->second.failed) return fail(DPF_EINVAL, "hash table %d failed to build", J.ht);
    int idx;
    dpf_status st = cs.add(J.fk_col, &idx);
    if (st) return st;
    const int codec = c->cols[J.fk_col].codec;
    if (codec != C_FOR && codec != C_DELTA) return fail(DPF_EINVAL, "join column %d must be FOR or DELTA", J.fk_col);
    DevStep S;
    std::memset(&S, 0, sizeof S);
    S.kind = ST_PROBE;
    S.col = uint8_t(idx);
    const HashTable& H = ht->second;
    S.ht_kind = uint8_t(H.kind);
    if (H.kind == HT_DIRECT || H.kind == HT_RANK) {
      S.ht = H.kind == HT_DIRECT ? static_cast<const void*>(H.direct) : static_cast<const void*>(H.rank);
      S.kmin = H.kmin;
      S.krange = H.capacity;
    } else {
      S.ht = H.slots;
      S.ht_mask = H.capacity - 1;
    }
    S.zlo = H.key_lo;
    S.zhi = H.key_hi;
    probe_step.push_back(steps.size());
    sel.push_back(step_selectivity(S, nullptr, &ht->second));
    steps.push_back(S);
    probes.push_back(&ht->second);
  }
  // group keys: dense ids in lexicographic (first key most significant) order
  uint64_t dom[2] = {1, 1};
  for (int k = 0; k < P.n_keys; ++k) {
    const dpf_key& K = P.keys[k];
    if (K.kind == DPF_KEY_COLUMN) {
      auto it = c->cols.find(K.col);
      if (it == c->cols.end() || it->second.codec != C_DICT) return fail(DPF_EINVAL, "group key column %d must be a DICT column", K.col);
      dom[k] = it->second.dict.size();
      Q.key_dict[k] = it->second.d_dict;
    } else if (K.kind == DPF_KEY_PAYLOAD) {
      if (K.join < 0 || K.join >= P.n_joins) return fail(DPF_EINVAL, "group key %d names join %d", k, K.join);
      const HashTable& h = *probes[K.join];
      if (K.field < 0 || K.field >= h.npay) return fail(DPF_EINVAL, "hash table %d has no payload field %d", h.id, K.field);
      dom[k] = h.pay_dom[K.field];
      Q.key_dict[k] = h.pay_dict[K.field];
    } else {
      return fail(DPF_EINVAL, "unknown key kind %d", K.kind);
    }
    if (dom[k] == 0) return fail(DPF_EINVAL, "group key %d has an empty domain", k);
  }
  const uint64_t domain = dom[0] * dom[1];
  if (domain > DPF_MAX_GROUPS) return fail(DPF_EINVAL, "group domain %llu exceeds %d", (unsigned long long)domain, DPF_MAX_GROUPS);
  Q.nkeys = uint32_t(P.n_keys);
  Q.domain = uint32_t(domain);
  for (int k = 0; k < 2; ++k) {
    Q.key_dom[k] = uint32_t(dom[k]);
    Q.key_div[k] = (k == 0 && P.n_keys == 2) ? uint32_t(dom[1]) : 1u;
  }
  for (int k = 0; k < P.n_keys; ++k) {
    const dpf_key& K = P.keys[k];
    if (K.kind == DPF_KEY_PAYLOAD) {
      DevStep& S = steps[probe_step[K.join]];
      if (K.field == 0) S.mul0 += Q.key_div[k]; else S.mul1 += Q.key_div[k];
    } else {
      int idx;
      dpf_status st = cs.add(K.col, &idx);
      if (st) return st;
      DevStep S;
      std::memset(&S, 0, sizeof S);
      S.kind = ST_KEY;
      S.col = uint8_t(idx);
      S.key_mul = Q.key_div[k];
      S.zlo = INT32_MIN;
      S.zhi = INT32_MAX;
      sel.push_back(step_selectivity(S, nullptr, nullptr));
      steps.push_back(S);
    }
  }
  Q.naggs = uint32_t(P.n_aggs);
  for (int a = 0; a < P.n_aggs; ++a) {
    const dpf_agg& A = P.aggs[a];
    if (A.op < DPF_AGG_COUNT || A.op > DPF_AGG_SUM_SUB) return fail(DPF_EINVAL, "unknown aggregate op %d", A.op);
    Q.agg_op[a] = uint8_t(A.op);
    const int need = A.op == DPF_AGG_COUNT ? 0 : (A.op == DPF_AGG_SUM ? 1 : 2);
    const dpf_col_id ab[2] = {A.a, A.b};
    for (int i = 0; i < need; ++i) {
      auto it = c->cols.find(ab[i]);
      if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown aggregate column %d", ab[i]);
      if (it->second.codec != C_FOR && it->second.codec != C_DELTA && it->second.codec != C_FOR64)
        return fail(DPF_EINVAL, "aggregate column %d must be FOR, DELTA or FOR64", ab[i]);
      int idx;
      dpf_status st = cs.add(ab[i], &idx);
      if (st) return st;
      (i == 0 ? Q.agg_a : Q.agg_b)[a] = uint8_t(idx);
    }
  }
  for (int32_t id : unread) {
    int idx;
    dpf_status st = cs.ids.empty() ? cs.add(id, &idx) : cs.check(id);
    if (st) return st;
  }
  if (cs.ids.empty() && P.scan_col != 0) {
    int idx;
    dpf_status st = cs.add(P.scan_col, &idx);
    if (st) return st;
  }
  if (cs.ids.empty()) return fail(DPF_EINVAL, "plan names no column of the scanned table");
  if (steps.size() > size_t(kMaxSteps)) return fail(DPF_EINVAL, "plan compiles to more than %d steps", kMaxSteps);
  // Step order from a small cost model (the result does not depend on it: a
  // conjunction, and group-id contributions add).  The first step runs
  // densely over the rows of the pages its zone map keeps (the pages whose
  // value bounds meet the step's range; the kernel skips the others
  // unread) at a cost of about its column's bits per row; every later step
  // runs over the survivors of the steps before it at about kSparseCost
  // bit-equivalents per survivor (a sector read and a probe).  For a given
  // first step, later filters go most selective first; group keys come
  // last.  The plan's own first filter is kept unless another first step is
  // estimated 5 % cheaper.
  constexpr double kSparseCost = 64.0;
  std::vector<size_t> filters, keys;
  for (size_t i = 0; i < steps.size(); ++i) (steps[i].kind == ST_KEY ? keys : filters).push_back(i);
  std::vector<double> bits(steps.size(), 32.0);
  for (size_t i = 0; i < steps.size(); ++i) {
    const Column& col = c->cols[cs.ids[steps[i].col]];
    if (col.nrows) bits[i] = 8.0 * double(col.bytes) / double(col.nrows) + (steps[i].kind == ST_PROBE ? 4.0 : 0.0);
    bits[i] *= zone_fraction(col, steps[i].zlo, steps[i].zhi);
  }
  auto plan_cost = [&](size_t first, std::vector<size_t>* out) {
    std::vector<size_t> rest;
    for (size_t i : filters)
      if (i != first) rest.push_back(i);
    std::stable_sort(rest.begin(), rest.end(), [&](size_t a, size_t b) { return sel[a] < sel[b]; });
    double cost = bits[first], surv = std::min(1.0, sel[first]);
    for (size_t i : rest) {
      cost += surv * kSparseCost;
      surv *= std::min(1.0, sel[i]);
    }
    cost += surv * kSparseCost * double(keys.size());
    if (out) {
      out->assign(1, first);
      out->insert(out->end(), rest.begin(), rest.end());
      out->insert(out->end(), keys.begin(), keys.end());
    }
    return cost;
  };
  // A 64-bit range (a FOR64 column) runs only over survivors, never as the
  // dense first step; when every filter is one, a pass-all first step that
  // reads nothing leads.
  std::vector<size_t> leads;
  for (size_t f : filters)
    if (!is_step64(steps[f].kind)) leads.push_back(f);
  if (!filters.empty() && leads.empty()) {
    DevStep A;
    std::memset(&A, 0, sizeof A);
    A.kind = ST_ALL;
    A.col = steps[filters[0]].col;
    A.zlo = INT32_MIN;
    A.zhi = INT32_MAX;
    steps.push_back(A);
    sel.push_back(1.0);
    bits.push_back(0.0);
    leads.push_back(steps.size() - 1);
    filters.push_back(steps.size() - 1);
    if (steps.size() > size_t(kMaxSteps)) return fail(DPF_EINVAL, "plan compiles to more than %d steps", kMaxSteps);
  }
  std::vector<size_t> order(steps.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  if (!filters.empty()) {
    size_t best = leads[0];
    double best_cost = plan_cost(best, nullptr);
    const double own = best_cost;
    for (size_t f : leads) {
      const double cst = plan_cost(f, nullptr);
      if (cst < best_cost && cst < 0.95 * own) {
        best = f;
        best_cost = cst;
      }
    }
    plan_cost(best, &order);
  }
  Q.nsteps = uint32_t(steps.size());
  for (size_t i = 0; i < steps.size(); ++i) Q.steps[i] = steps[order[i]];
  // When the first step keeps enough rows (>= 3 % estimated), most 32-byte
  // sectors of step 1's column hold a survivor's field anyway: prefetch its
  // mini blocks into L2 while the dense tiles run, so that step's
  // per-survivor reads hit L2 instead of waiting on DRAM.
  if (steps.size() > 1 && sel[order[0]] >= kPrefetchMinSel && Q.steps[1].kind != ST_PREFIX &&
      Q.steps[1].kind != ST_CONTAINS && Q.steps[1].kind != ST_LIKE && !is_step64(Q.steps[1].kind) &&
      Q.steps[0].kind != ST_ALL)
    Q.pf_step = 1;
  Q.nrows = cs.nrows;
  Q.page_rows = cs.page_rows;
  *host = cs.host;
  return DPF_OK;
}

// Places join tables in the CTA's shared-memory region while they fit the
// budget: open-addressing tables as 8-byte slots, direct tables as 1/2/4-byte
// group-id contributions.  With first_only, only a table probed by the first
// (dense) step is a candidate: that step probes every row, so its lookups
// gain most from shared memory, while later steps probe few survivors and
// their tables serve from L1/L2 without taking shared memory from the other
// resident CTAs.  Returns the bytes used.
size_t place_tables(DevQuery& Q, size_t budget, bool first_only) {
  const uint32_t width = Q.domain <= 255 ? 1u : (Q.domain <= 65535 ? 2u : 4u);
  size_t used = 0;
  // PREFIX / CONTAINS steps on FSST columns: the code-level matcher tables
  // (fsst_match_bytes), whichever step they are, while they fit
  for (uint32_t s = 0; s < Q.nsteps; ++s) {
    DevStep& S = Q.steps[s];
    if ((S.kind != ST_PREFIX && S.kind != ST_CONTAINS) || Q.cols[S.col].codec != C_FSST) continue;
    S.smem_width = 0;
    if (S.plen == 0) continue;
    const size_t bytes = fsst_match_bytes(S.plen);
    const size_t at = (used + 15) & ~size_t(15);
    if (at + bytes > budget) continue;
    S.smem_width = 1;
    S.smem_off = uint32_t(at);
    used = at + bytes;
  }
  for (uint32_t s = 0; s < Q.nsteps; ++s) {
    DevStep& S = Q.steps[s];
    if (S.kind != ST_PROBE) continue;
    S.smem_width = 0;
    if (first_only && s != 0) continue;
    if (S.ht_kind == HT_RANK) continue;  // probed in device memory (L2) only
    const uint32_t w = S.ht_kind == HT_DIRECT ? width : 8u;
    const size_t bytes = S.ht_kind == HT_DIRECT ? size_t(S.krange) * w : size_t(S.ht_mask + 1) * 8;
    const size_t at = (used + 15) & ~size_t(15);
    if (at + bytes > budget) continue;
    S.smem_width = uint8_t(w);
    S.smem_off = uint32_t(at);
    used = at + bytes;
  }
  used = (used + 15) & ~size_t(15);
  Q.smem_table_bytes = uint32_t(used);
  return used;
}

// Signature of a set of plans for the tuning cache: what the launch
// configuration's speed depends on (rows and encoding of every column a plan
// reads, its steps, join tables, groups and aggregates), not the predicate
// constants.  FNV-1a over those fields.
uint64_t plans_signature(dpf_ctx* c, const dpf_plan* plans, int32_t n) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) {
    for (int i = 0; i < 8; ++i) {
      h ^= (x >> (8 * i)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  auto col = [&](dpf_col_id id) {
    auto it = c->cols.find(id);
    if (it == c->cols.end()) return mix(~0ull);
    mix(it->second.nrows);
    mix(uint64_t(it->second.codec) << 32 | it->second.page_rows);
    mix(it->second.bytes);
  };
  mix(uint64_t(n));
  for (int32_t i = 0; i < n; ++i) {
    const dpf_plan& P = plans[i];
    mix(uint64_t(P.n_preds) | uint64_t(P.n_joins) << 16 | uint64_t(P.n_keys) << 32 | uint64_t(P.n_aggs) << 48);
    col(P.scan_col);
    for (int k = 0; k < P.n_preds && P.preds; ++k) {
      col(P.preds[k].col);
      mix(uint64_t(P.preds[k].op));
    }
    for (int k = 0; k < P.n_joins && P.joins; ++k) {
      col(P.joins[k].fk_col);
      auto it = c->hts.find(P.joins[k].ht);
      mix(it == c->hts.end() ? ~0ull : (uint64_t(it->second.kind) << 32 | it->second.capacity));
    }
    for (int k = 0; k < P.n_keys && P.keys; ++k) mix(uint64_t(P.keys[k].kind) << 32 | uint32_t(P.keys[k].col));
    for (int k = 0; k < P.n_aggs && P.aggs; ++k) {
      mix(uint64_t(P.aggs[k].op));
      col(P.aggs[k].a);
      if (P.aggs[k].op >= DPF_AGG_SUM_MUL) col(P.aggs[k].b);
    }
  }
  return h;
}

// Fields left 0 take the tuning dpf_autotune stored for these plans, else the
// defaults.
void fill_tuning_defaults(dpf_ctx* c, dpf_tuning& t, const dpf_plan* plans, int32_t n) {
  if (t.chunk_rows == 0 || t.threads == 0 || t.ht_placement == 0 || t.ctas_per_sm == 0 || t.staging == 0 ||
      t.group_agg == 0) {
    auto it = c->tune_cache.find(plans_signature(c, plans, n));
    if (it != c->tune_cache.end()) {
      if (t.chunk_rows == 0) t.chunk_rows = it->second.chunk_rows;
      if (t.threads == 0) t.threads = it->second.threads;
      if (t.ht_placement == 0) t.ht_placement = it->second.ht_placement;
      if (t.ctas_per_sm == 0) t.ctas_per_sm = it->second.ctas_per_sm;
      if (t.staging == 0) t.staging = it->second.staging;
      if (t.group_agg == 0) t.group_agg = it->second.group_agg;
    }
  }
  const dpf_tuning& d = c->defaults;  // the context's defaults (dpf_set_tuning)
  if (t.chunk_rows == 0) t.chunk_rows = d.chunk_rows;
  if (t.threads == 0) t.threads = d.threads;
  if (t.ht_placement == 0) t.ht_placement = d.ht_placement;
  if (t.ctas_per_sm == 0) t.ctas_per_sm = d.ctas_per_sm;
  if (t.staging == 0) t.staging = d.staging;
  if (t.group_agg == 0) t.group_agg = d.group_agg;
  if (t.chunk_rows == 0) t.chunk_rows = kDefaultChunkRows;
  if (t.threads == 0) t.threads = 256;
  if (t.ht_placement == 0) t.ht_placement = DPF_HT_AUTO;
  if (t.staging == 0) t.staging = kDefaultStaging;
  if (t.group_agg == 0) t.group_agg = kDefaultGroupAgg;
}

// A flat JSON object of launch-configuration fields (dpf_set_tuning): the
// keys of dpf_tuning with non-negative integers, or for the three enums
// their names ("auto" / "smem" / "global", "default" / "on" / "off",
// "default" / "warp" / "atomic").  Returns false on anything else.
bool parse_tuning_json(const char* js, dpf_tuning* out, std::string* why) {
  dpf_tuning t{};
  const char* p = js;
  auto ws = [&] { while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p; };
  auto str = [&](std::string* v) {
    if (*p != '"') return false;
    ++p;
    v->clear();
    while (*p && *p != '"') {
      if (*p == '\\' || v->size() > 32) return false;
      v->push_back(*p++);
    }
    if (*p != '"') return false;
    ++p;
    return true;
  };
  ws();
  if (*p != '{') { *why = "expected '{'"; return false; }
  ++p;
  ws();
  bool first = true;
  while (*p != '}') {
    if (!first) {
      if (*p != ',') { *why = "expected ',' or '}'"; return false; }
      ++p;
      ws();
    }
    first = false;
    std::string key, sval;
    if (!str(&key)) { *why = "expected a quoted key"; return false; }
    ws();
    if (*p != ':') { *why = "expected ':' after \"" + key + "\""; return false; }
    ++p;
    ws();
    int64_t num = -1;
    if (*p == '"') {
      if (!str(&sval)) { *why = "bad string value for \"" + key + "\""; return false; }
    } else if (*p >= '0' && *p <= '9') {
      num = 0;
      while (*p >= '0' && *p <= '9') {
        num = num * 10 + (*p++ - '0');
        if (num > (int64_t(1) << 31)) { *why = "value of \"" + key + "\" too large"; return false; }
      }
    } else {
      *why = "value of \"" + key + "\" must be a non-negative integer or a name";
      return false;
    }
    ws();
    auto pick = [&](std::initializer_list<const char*> names, int32_t* dst) {
      if (num >= 0) {
        if (num >= int64_t(names.size())) return false;
        *dst = int32_t(num);
        return true;
      }
      int32_t i = 0;
      for (const char* nm : names) {
        if (sval == nm) { *dst = i; return true; }
        ++i;
      }
      return false;
    };
    bool ok = true;
    if (key == "chunk_rows") {
      ok = num >= 0 && num % 512 == 0 && num <= (int64_t(1) << 24);
      t.chunk_rows = uint32_t(num);
    } else if (key == "threads") {
      ok = num == 0 || num == 128 || num == 256 || num == 512 || num == 1024;
      t.threads = uint32_t(num);
    } else if (key == "ctas_per_sm") {
      ok = num >= 0 && num <= 32;
      t.ctas_per_sm = uint32_t(num);
    } else if (key == "ht_placement") {
      ok = pick({"auto", "smem", "global"}, &t.ht_placement);
    } else if (key == "staging") {
      ok = pick({"default", "on", "off"}, &t.staging);
    } else if (key == "group_agg") {
      ok = pick({"default", "warp", "atomic"}, &t.group_agg);
    } else {
      *why = "unknown key \"" + key + "\"";
      return false;
    }
    if (!ok) { *why = "bad value for \"" + key + "\""; return false; }
  }
  ++p;
  ws();
  if (*p) { *why = "text after the object"; return false; }
  *out = t;
  return true;
}

dpf_status release_prep(dpf_ctx* c, Prep* p) {
  if (p->launched && p->ev) cudaEventSynchronize(p->ev);
  for (HashTable* h : p->chain) --h->refs;
  p->chain.clear();
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->ev) cudaEventDestroy(p->ev);
  dev_free(c, p->dq);
  dev_free(c, p->dqbegin);
  dev_free(c, p->sched);
  dev_free(c, p->scratch);
  dev_free(c, p->unf_scratch);
  return DPF_OK;
}

// Launch of a prepared batch (fused kernel or unfused chain) on s.
cudaError_t launch_prep(Prep* p, cudaStream_t s) {
  for (HashTable* h : p->chain) {
    const cudaError_t e = enqueue_table_build(*h, s);
    if (e != cudaSuccess) return e;
    h->pending = true;
  }
  if (p->unfused) {
    uint32_t n = 0;
    cudaError_t e = launch_unfused(p->U, s, &n);
    p->launches = n;
    return e;
  }
  return launch_fused(p->L, s);
}

dpf_status prepare(dpf_ctx* c, const dpf_plan* plans, int32_t n, const dpf_tuning* tuning, Prep** out) {
  if (!plans || n < 1 || n > 4096) return fail(DPF_EINVAL, "need 1..4096 plans");
  auto p = std::make_unique<Prep>();
  p->nq = n;
  p->hq.resize(size_t(n));
  dpf_tuning t{};
  if (tuning) t = *tuning;
  fill_tuning_defaults(c, t, plans, n);
  if (t.chunk_rows % (kMbPerWarpTile * kMB) != 0 || t.chunk_rows > (1u << 24))
    return fail(DPF_EINVAL, "chunk_rows %u must be a multiple of %u and at most 2^24", t.chunk_rows, kMbPerWarpTile * kMB);
  if (t.threads != 128 && t.threads != 256 && t.threads != 512 && t.threads != 1024)
    return fail(DPF_EINVAL, "threads must be 128, 256, 512 or 1024");
  if (t.staging != DPF_STAGE_ON && t.staging != DPF_STAGE_OFF) return fail(DPF_EINVAL, "staging must be 0, 1 or 2");
  if (t.group_agg != DPF_GROUP_AGG_WARP && t.group_agg != DPF_GROUP_AGG_ATOMIC)
    return fail(DPF_EINVAL, "group_agg must be 0, 1 or 2");
  bool any_warp_agg = false;
  bool host = false;
  uint64_t tickets = 0;
  std::vector<uint64_t> qbegin(size_t(n) + 1);
  // scratch layout per query: acc | done | out_n | out
  std::vector<uint64_t> off_acc(n), off_done(n), off_outn(n), off_out(n);
  uint64_t scratch = 0;
  size_t max_tables = 0;
  uint32_t acc_slots = 0;
  // SMEM placement: what the opt-in shared memory leaves after the largest
  // accumulator region, the warps' lists and group buffers, and the plan
  const int per_cta_fixed = int(kSmemAccSlots * 8) + int(t.threads / 32) * int(kListBytesPerWarp) + 4096;
  const size_t table_budget =
      t.ht_placement == DPF_HT_GLOBAL ? 0
      : t.ht_placement == DPF_HT_SMEM ? size_t(std::max(0, c->smem_optin - per_cta_fixed))
                                      : size_t(48 * 1024);
  for (int i = 0; i < n; ++i) {
    DevQuery& Q = p->hq[i];
    bool h = false;
    std::vector<const HashTable*> probes;
    dpf_status st = compile_plan(c, plans[i], Q, &h, probes);
    if (st) return fail(st, "plan %d: %s", i, t_last_error.c_str());
    host |= h;
    const size_t used = place_tables(Q, table_budget, t.ht_placement == DPF_HT_AUTO);
    max_tables = std::max(max_tables, used);
    Q.chunk_rows = t.chunk_rows;
    Q.nchunks = (Q.nrows + t.chunk_rows - 1) / t.chunk_rows;
    Q.chunk_begin = tickets;
    qbegin[i] = tickets;
    tickets += Q.nchunks;
    const uint32_t S1 = 1 + Q.naggs;
    Q.use_smem_acc = uint64_t(Q.domain) * S1 <= kSmemAccSlots ? 1u : 0u;
    Q.warp_agg = t.group_agg == DPF_GROUP_AGG_WARP && Q.domain > 1 ? 1u : 0u;
    any_warp_agg = any_warp_agg || Q.warp_agg;
    if (Q.use_smem_acc) acc_slots = std::max<uint32_t>(acc_slots, Q.domain * S1);
    off_acc[i] = scratch; scratch += align16(uint64_t(Q.domain) * S1 * 8);
    off_done[i] = scratch; scratch += 16;
    off_outn[i] = scratch; scratch += 16;
    off_out[i] = scratch; scratch += align16(uint64_t(std::max<uint32_t>(Q.domain, 1)) * sizeof(dpf_record));
  }
  qbegin[n] = tickets;
  // Staging ring: a launch stages all of its queries or none; a query can be
  // staged when its first step is an integer step over device-resident
  // pages.  The ring's slots are as wide as the widest mini block of those
  // steps' columns.
  uint32_t stage_bw = 0;
  bool text = false;
  for (const DevQuery& q : p->hq) text = text || needs_string_matcher(q);
  if (t.staging == DPF_STAGE_ON && !host && !text) {
    bool all = true;
    for (const DevQuery& Q : p->hq) {
      const DevStep& S0 = Q.steps[0];
      const DevColumn& C0 = Q.cols[S0.col];
      const bool ok = Q.nsteps != 0 && S0.kind != ST_PREFIX && S0.kind != ST_CONTAINS && S0.kind != ST_LIKE &&
                      S0.kind != ST_ALL &&
                      (C0.codec == C_FOR || C0.codec == C_DICT || C0.codec == C_DELTA) && C0.max_bw <= 32;
      all = all && ok;
      if (ok) stage_bw = std::max(stage_bw, std::max<uint32_t>(C0.max_bw, 1u));
    }
    if (!all) stage_bw = 0;
    for (DevQuery& Q : p->hq) Q.stage = stage_bw;
  }
  if (t.threads > 256 && (host || text || stage_bw))
    return fail(DPF_EINVAL, "CTAs of %u threads run device-resident batches without string-matcher steps, unstaged",
                t.threads);
  dpf_status st;
  if ((st = dev_alloc(c, scratch, reinterpret_cast<void**>(&p->scratch)))) return st;
  if ((st = dev_alloc_t(c, uint64_t(n), &p->dq)) || (st = dev_alloc_t(c, uint64_t(n) + 1, &p->dqbegin)) ||
      (st = dev_alloc_t(c, 1, &p->sched))) {
    release_prep(c, p.get());
    return st;
  }
  for (int i = 0; i < n; ++i) {
    DevQuery& Q = p->hq[i];
    Q.acc = reinterpret_cast<unsigned long long*>(p->scratch + off_acc[i]);
    Q.done = reinterpret_cast<unsigned int*>(p->scratch + off_done[i]);
    Q.out_n = reinterpret_cast<unsigned int*>(p->scratch + off_outn[i]);
    Q.out = p->scratch + off_out[i];
  }
  cudaError_t e = cudaMemsetAsync(p->scratch, 0, scratch, c->io);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->sched, 0, sizeof(Sched), c->io);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->dq, p->hq.data(), sizeof(DevQuery) * n, cudaMemcpyHostToDevice, c->io);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->dqbegin, qbegin.data(), 8 * (n + 1), cudaMemcpyHostToDevice, c->io);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->io);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release_prep(c, p.get());
    return fail(DPF_ECUDA, "prepare: %s", cudaGetErrorString(e));
  }
  // ctas_per_sm >= 4 selects the kernel build for four resident CTAs per SM
  // (64 registers) when four fit; otherwise the build for three (80)
  int min_blocks = kFusedMinBlocksLo;
  int per_sm = 0;
  if (t.ctas_per_sm >= uint32_t(kFusedMinBlocksHi)) {
    per_sm = fused_blocks_per_sm(int(t.threads), acc_slots, max_tables, host, kFusedMinBlocksHi, stage_bw);
    if (per_sm >= kFusedMinBlocksHi * 256 / int(t.threads)) min_blocks = kFusedMinBlocksHi;
  }
  if (min_blocks == kFusedMinBlocksLo)
    per_sm = fused_blocks_per_sm(int(t.threads), acc_slots, max_tables, host, kFusedMinBlocksLo, stage_bw);
  if (per_sm < 1) {
    release_prep(c, p.get());
    return fail(DPF_EINVAL, "fused kernel does not fit on an SM with %u threads and %zu table bytes", t.threads, max_tables);
  }
  if (t.ctas_per_sm == 0 || int(t.ctas_per_sm) > per_sm || min_blocks == kFusedMinBlocksHi) t.ctas_per_sm = uint32_t(per_sm);
  // Tickets are handed out in order, so the launch ends on the last query's
  // last tickets.  Whole-size tickets there leave most warps idle while the
  // last few finish; the final rows (about two tickets of tail_rows per warp
  // of the grid, taken from the last queries backwards) are cut into tickets
  // of chunk_rows / 8 rows instead.  In a batch the same holds at every query
  // switch: a CTA's warps meet when their tickets leave a query (its plan,
  // tables and accumulators sit in shared memory), so each query's last rows
  // (one small ticket per warp of the grid) are cut small as well.
  {
    const uint64_t warps = uint64_t(c->num_sms) * t.ctas_per_sm * (t.threads / 32);
    const uint32_t tile_rows = kMbPerWarpTile * kMB;
    const uint32_t tail_rows = std::max<uint32_t>(tile_rows, t.chunk_rows / 8 / tile_rows * tile_rows);
    std::vector<uint64_t> tail_len(size_t(n), 0);
    if (tail_rows < t.chunk_rows) {
      if (n > 1)
        for (int i = 0; i < n; ++i) tail_len[size_t(i)] = std::min<uint64_t>(p->hq[i].nrows, warps * tail_rows);
      uint64_t want = 2 * warps * tail_rows;
      for (int i = n - 1; i >= 0 && want > 0; --i) {
        const uint64_t rows = std::min<uint64_t>(p->hq[i].nrows, want);
        tail_len[size_t(i)] = std::max(tail_len[size_t(i)], rows);
        want -= rows;
      }
    }
    for (int i = 0; i < n; ++i) {
      DevQuery& Q = p->hq[i];
      if (tail_len[size_t(i)] == 0) continue;
      const uint64_t keep_big = (Q.nrows - tail_len[size_t(i)]) / t.chunk_rows;
      Q.tail_first = keep_big;
      Q.tail_rows = tail_rows;
      const uint64_t tail = Q.nrows - keep_big * t.chunk_rows;
      Q.nchunks = keep_big + (tail + tail_rows - 1) / tail_rows;
    }
    tickets = 0;
    for (int i = 0; i < n; ++i) {
      p->hq[i].chunk_begin = tickets;
      qbegin[i] = tickets;
      tickets += p->hq[i].nchunks;
    }
    qbegin[n] = tickets;
    e = cudaMemcpyAsync(p->dq, p->hq.data(), sizeof(DevQuery) * n, cudaMemcpyHostToDevice, c->io);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->dqbegin, qbegin.data(), 8 * (n + 1), cudaMemcpyHostToDevice, c->io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->io);
    if (e != cudaSuccess) {
      release_prep(c, p.get());
      return fail(DPF_ECUDA, "prepare: %s", cudaGetErrorString(e));
    }
  }
  p->L.min_blocks = min_blocks;
  p->tuning = t;
  p->L.queries = p->dq;
  p->L.qbegin = p->dqbegin;
  p->L.nq = n;
  p->L.total_chunks = tickets;
  p->L.sched = p->sched;
  p->L.threads = int(t.threads);
  p->L.grid = int(std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(c->num_sms) * t.ctas_per_sm, tickets)));
  p->L.smem_tables = max_tables;
  p->L.acc_slots = acc_slots;
  p->L.host_data = host;
  p->L.stage_bw = stage_bw;
  p->tuning.staging = stage_bw ? DPF_STAGE_ON : DPF_STAGE_OFF;  // what the launch does
  p->tuning.group_agg = any_warp_agg ? DPF_GROUP_AGG_WARP : DPF_GROUP_AGG_ATOMIC;
  p->L.text = false;
  for (const DevQuery& q : p->hq) p->L.text = p->L.text || needs_string_matcher(q);
  p->fetched.assign(size_t(n), 0);
  p->id = c->next_prep++;
  *out = p.get();
  c->preps[p->id] = std::move(p);
  return DPF_OK;
}

Prep* find_prep(dpf_ctx* c, dpf_prep_id id) {
  auto it = c->preps.find(id);
  return it == c->preps.end() ? nullptr : it->second.get();
}

dpf_status wait_event(cudaEvent_t ev, int32_t timeout_ms) {
  if (timeout_ms < 0) {
    CUDA_TRY(cudaEventSynchronize(ev));
    return DPF_OK;
  }
  const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return DPF_OK;
    if (e != cudaErrorNotReady) return fail(DPF_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
    if (std::chrono::steady_clock::now() >= until) return fail(DPF_ETIMEOUT, "result not ready within %d ms", timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

dpf_status read_result(dpf_ctx* c, Prep* p, int32_t i, dpf_record* buf, uint64_t cap, uint64_t* n_out,
                       int32_t timeout_ms) {
  if (i < 0 || i >= p->nq) return fail(DPF_EINVAL, "query index %d out of range", i);
  if (!p->launched) return fail(DPF_EINVAL, "batch %d was never launched", p->id);
  dpf_status st = wait_event(p->ev, timeout_ms);
  if (st) return st;
  uint32_t status = 0, n = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, &p->sched->status, 4, cudaMemcpyDeviceToHost, c->io));
  CUDA_TRY(cudaMemcpyAsync(&n, p->hq[i].out_n, 4, cudaMemcpyDeviceToHost, c->io));
  CUDA_TRY(cudaStreamSynchronize(c->io));
  if (status) {
    cudaMemsetAsync(&p->sched->status, 0, 4, c->io);
    cudaStreamSynchronize(c->io);
    if (status & S_CORRUPT) return fail(DPF_ECORRUPT, "device reported corrupt data (status %u)", status);
    return fail(DPF_EINTERNAL, "device reported an internal error (status %u)", status);
  }
  if (n_out) *n_out = n;
  if (cap < n) return fail(DPF_ETRUNC, "need %u records", n);
  if (n) {
    if (!buf) return fail(DPF_EINVAL, "buf is NULL");
    CUDA_TRY(cudaMemcpyAsync(buf, p->hq[i].out, uint64_t(n) * sizeof(dpf_record), cudaMemcpyDeviceToHost, c->io));
    CUDA_TRY(cudaStreamSynchronize(c->io));
  }
  return DPF_OK;
}

}  // namespace

namespace dpf {

// Compiles one plan for dpf_execute_noalloc (no device allocation): the
// device plan with hash tables placed in shared memory as dpf_prepare's
// automatic placement would, the table bytes and the launch geometry.
dpf_status noalloc_compile(dpf_ctx* c, const dpf_plan* plan, DevQuery* Q, size_t* smem_tables, bool* host,
                           int* device, int* num_sms) {
  std::vector<const HashTable*> probes;
  dpf_status st = compile_plan(c, *plan, *Q, host, probes);
  if (st) return st;
  const size_t used = place_tables(*Q, size_t(48 * 1024), true);
  *smem_tables = used;
  *device = c->device;
  *num_sms = c->num_sms;
  return DPF_OK;
}

std::recursive_mutex& ctx_mutex(dpf_ctx* c) { return c->mu; }

}  // namespace dpf

// ======================================================================
// C ABI
// ======================================================================
extern "C" {

const char* dpf_last_error(void) { return t_last_error.c_str(); }

dpf_status dpf_create(dpf_ctx** out, int32_t device, uint64_t hbm_budget, const dpf_alloc_hooks* hooks) {
  if (!out) return fail(DPF_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(DPF_ECUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return fail(DPF_EINVAL, "device %d out of range (%d devices)", device, ndev);
  if (hooks && (!hooks->alloc || !hooks->free)) return fail(DPF_EINVAL, "hooks need alloc and free");
  DeviceGuard g(device);
  auto c = std::make_unique<dpf_ctx>();
  c->device = device;
  c->budget = hbm_budget;
  if (hooks) {
    c->hooks = *hooks;
    c->has_hooks = true;
  }
  CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  CUDA_TRY(cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  CUDA_TRY(cudaStreamCreateWithFlags(&c->io, cudaStreamNonBlocking));
  dpf_status st;
  if ((st = dev_alloc_t(c.get(), 1, &c->bsched)) || (st = dev_alloc_t(c.get(), 1, &c->bcount)) ||
      (st = dev_alloc_t(c.get(), 2, &c->bkminmax)))
    return st;
  CUDA_TRY(cudaMemsetAsync(c->bsched, 0, sizeof(Sched), c->io));
  CUDA_TRY(cudaStreamSynchronize(c->io));
  *out = c.release();
  return DPF_OK;
}

dpf_status dpf_destroy(dpf_ctx* c) {
  if (!c) return DPF_OK;
  {
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (auto& kv : c->preps) release_prep(c, kv.second.get());
    c->preps.clear();
    for (auto& kv : c->hts) free_table(c, kv.second);
    for (auto& kv : c->cols) free_column(c, kv.second);
    dev_free(c, c->bsched);
    dev_free(c, c->bcount);
    dev_free(c, c->bkminmax);
    drop_cache(c);
    if (c->io) cudaStreamDestroy(c->io);
  }
  delete c;
  return DPF_OK;
}

dpf_status dpf_memory_used(dpf_ctx* c, uint64_t* bytes) {
  if (!c || !bytes) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  *bytes = c->used;
  return DPF_OK;
}

dpf_status dpf_load_encoded(dpf_ctx* c, const dpf_column_desc* d, const uint8_t* pages, uint64_t size,
                            const uint64_t* page_off, const uint64_t* row_prefix, uint64_t nrows,
                            const int32_t* dict, uint64_t dict_n, dpf_col_id* out) {
  if (!c || !d || !pages || !page_off || !row_prefix || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  const uint32_t codec = uint32_t(d->codec);
  const uint32_t P = d->page_rows ? d->page_rows : kDefaultPageRows;
  if (codec < C_FOR || codec > C_FOR64) return fail(DPF_EINVAL, "unknown codec %u", codec);
  if (nrows == 0 || P % kMB || P > kMaxPageRows) return fail(DPF_EINVAL, "bad nrows or page_rows");
  if (codec == C_FSST) {
    if (!dict || dict_n == 0 || dict_n % 3 || dict_n / 3 > kFsstMaxSymbols)
      return fail(DPF_EINVAL, "FSST column needs a table of 1..255 symbols (3 int32 each)");
    for (uint64_t i = 0; i < dict_n / 3; ++i)
      if (dict[3 * i + 2] < 1 || dict[3 * i + 2] > 8) return fail(DPF_EINVAL, "FSST symbol %llu has length %d", (unsigned long long)i, dict[3 * i + 2]);
  }
  if (d->placement != DPF_PLACE_DEVICE && d->placement != DPF_PLACE_HOST_PINNED) return fail(DPF_EINVAL, "bad placement");
  if (codec == C_DICT && (!dict || dict_n == 0 || dict_n > 65536)) return fail(DPF_EINVAL, "DICT column needs 1..65536 dictionary values");
  if (codec == C_DICT)
    for (uint64_t i = 1; i < dict_n; ++i)
      if (dict[i] <= dict[i - 1]) return fail(DPF_EINVAL, "dictionary must be strictly ascending");
  const uint64_t npages = (nrows + P - 1) / P;
  for (uint64_t p = 0; p < npages; ++p)
    if (row_prefix[p] != std::min<uint64_t>(nrows, (p + 1) * uint64_t(P)))
      return fail(DPF_ECORRUPT, "RID index entry %llu is inconsistent", (unsigned long long)p);
  dpf_status st = validate_pages(codec, pages, size, page_off, npages, nrows, P, dict_n);
  if (st) return st;
  if (codec == C_FSST && (st = validate_fsst_codes(pages, page_off, npages, nrows, P, uint32_t(dict_n / 3)))) return st;
  Column col;
  col.codec = int32_t(codec);
  col.placement = d->placement;
  col.table = d->table;
  col.page_rows = P;
  col.nrows = nrows;
  col.npages = npages;
  col.bytes = size;
  col.page_off.assign(page_off, page_off + npages + 1);
  col.row_prefix.assign(row_prefix, row_prefix + npages);
  if (codec == C_DICT) col.dict.assign(dict, dict + dict_n);
  std::vector<int2> zones;
  value_bounds(codec, pages, page_off, npages, nrows, P, &col.vmin, &col.vmax, &zones, &col.max_bw);
  if (is_str_codec(codec)) {
    uint64_t sb = 0;
    for (uint64_t p = 0; p < npages; ++p) {
      const uint8_t* pg = pages + page_off[p];
      sb += page_off[p + 1] - page_off[p] - rd32(pg + 12);
    }
    col.raw_bytes = sb + 8 * nrows;
  } else {
    col.raw_bytes = (codec == C_FOR64 ? 8 : 4) * nrows;
  }
  if (col.placement == DPF_PLACE_HOST_PINNED) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&col.host_blob), size, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DPF_ENOMEM, "cudaHostAlloc(%llu): %s", (unsigned long long)size, cudaGetErrorString(e));
    }
    std::memcpy(col.host_blob, pages, size);
    void* dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, col.host_blob, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(col.host_blob);
      return fail(DPF_ECUDA, "cudaHostGetDevicePointer: %s", cudaGetErrorString(e));
    }
    col.blob = static_cast<uint8_t*>(dp);
  } else {
    void* dp;
    if ((st = dev_alloc(c, size, &dp))) return st;
    col.blob = static_cast<uint8_t*>(dp);
    if ((st = upload(c, col.blob, pages, size))) { free_column(c, col); return st; }
  }
  if ((st = dev_alloc_t(c, npages + 1, &col.d_page_off)) || (st = upload(c, col.d_page_off, page_off, 8 * (npages + 1))) ||
      (st = dev_alloc_t(c, std::max<uint64_t>(npages, 1), &col.d_zone)) ||
      (st = upload(c, col.d_zone, zones.data(), sizeof(int2) * npages))) {
    free_column(c, col);
    return st;
  }
  col.zones = std::move(zones);
  if (codec == C_DICT) {
    if ((st = dev_alloc_t(c, dict_n, &col.d_dict)) || (st = upload(c, col.d_dict, dict, 4 * dict_n))) {
      free_column(c, col);
      return st;
    }
  }
  if (codec == C_FSST) {
    col.nsym = dict_n / 3;
    std::vector<int4> sym(dict_n / 3);
    for (uint64_t i = 0; i < sym.size(); ++i) sym[i] = make_int4(dict[3 * i], dict[3 * i + 1], dict[3 * i + 2], 0);
    if ((st = dev_alloc_t(c, sym.size(), &col.d_sym)) || (st = upload(c, col.d_sym, sym.data(), sizeof(int4) * sym.size()))) {
      free_column(c, col);
      return st;
    }
  }
  col.id = c->next_col++;
  *out = col.id;
  c->cols[col.id] = std::move(col);
  return DPF_OK;
}

dpf_status dpf_load_column(dpf_ctx* c, const dpf_column_desc* d, const void* values, const uint64_t* str_offsets,
                           uint64_t nrows, dpf_col_id* out) {
  if (!c || !d || !out) return fail(DPF_EINVAL, "NULL argument");
  const uint32_t P = d->page_rows ? d->page_rows : kDefaultPageRows;
  if (nrows == 0 || P == 0) return fail(DPF_EINVAL, "nrows must be > 0");
  const uint64_t npages = (nrows + P - 1) / P;
  std::vector<uint64_t> page_off(npages + 1), row_prefix(npages);
  uint64_t size = 0, dict_n = 0;
  dpf_status st = dpf_encode_column(d, values, str_offsets, nrows, nullptr, 0, page_off.data(), row_prefix.data(),
                                    nullptr, 0, &dict_n, &size);
  if (st) return st;
  std::vector<uint8_t> pages(size);
  std::vector<int32_t> dict(std::max<uint64_t>(dict_n, 1));
  st = dpf_encode_column(d, values, str_offsets, nrows, pages.data(), size, page_off.data(), row_prefix.data(),
                         dict.data(), dict.size(), &dict_n, &size);
  if (st) return st;
  return dpf_load_encoded(c, d, pages.data(), size, page_off.data(), row_prefix.data(), nrows,
                          (d->codec == C_DICT || d->codec == C_FSST) ? dict.data() : nullptr, dict_n, out);
}

dpf_status dpf_column_info(dpf_ctx* c, dpf_col_id id, uint64_t* rows, uint64_t* enc, uint64_t* raw) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->cols.find(id);
  if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", id);
  if (rows) *rows = it->second.nrows;
  if (enc) *enc = it->second.bytes;
  if (raw) *raw = it->second.raw_bytes;
  return DPF_OK;
}

dpf_status dpf_column_read(dpf_ctx* c, dpf_col_id id, uint64_t offset, uint64_t bytes, uint8_t* host_out) {
  if (!c || (!host_out && bytes)) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->cols.find(id);
  if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", id);
  const Column& col = it->second;
  if (offset > col.bytes || bytes > col.bytes - offset) return fail(DPF_EINVAL, "range beyond the column");
  if (col.placement == DPF_PLACE_HOST_PINNED) {
    std::memcpy(host_out, col.host_blob + offset, bytes);
    return DPF_OK;
  }
  CUDA_TRY(cudaMemcpyAsync(host_out, col.blob + offset, bytes, cudaMemcpyDeviceToHost, c->io));
  CUDA_TRY(cudaStreamSynchronize(c->io));
  return DPF_OK;
}

dpf_status dpf_drop_column(dpf_ctx* c, dpf_col_id id) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->cols.find(id);
  if (it == c->cols.end()) return fail(DPF_EINVAL, "unknown column %d", id);
  cudaDeviceSynchronize();
  free_column(c, it->second);
  c->cols.erase(it);
  return DPF_OK;
}

// A hash build compiled on the host (Kernel #1 with no joins, Kernel #2
// with joins; Sec. 3.1): the scan's steps are the predicates in the given
// order, then one global-memory probe per join (a miss drops the row; no
// group-id contribution).  est_kept is the planner's estimate of the rows
// kept (the scanned rows times each step's estimated selectivity).
struct BuildSpec {
  DevQuery Q;
  HashTable ht;
  bool host = false;
  bool wide_payload = false;
  double est_kept = 0;
};

static dpf_status compile_build(dpf_ctx* c, const dpf_build& B, BuildSpec& bs) {
  if (B.n_payload < 0 || B.n_payload > 2 || (B.n_payload && !B.payload)) return fail(DPF_EINVAL, "0..2 payload fields");
  if (B.n_preds < 0 || B.n_preds > DPF_MAX_PREDS || (B.n_preds && !B.preds)) return fail(DPF_EINVAL, "bad predicates");
  if (B.n_joins < 0 || B.n_joins > DPF_MAX_JOINS || (B.n_joins && !B.joins)) return fail(DPF_EINVAL, "bad joins");
  DevQuery& Q = bs.Q;
  HashTable& ht = bs.ht;
  std::memset(&Q, 0, sizeof Q);
  ColumnSet cs{c, Q};
  const dpf_col_id key_col = B.key_col;
  int kidx;
  dpf_status st = cs.add(key_col, &kidx);
  if (st) return st;
  const Column& kc = c->cols[key_col];
  if (kc.codec != C_FOR && kc.codec != C_DELTA) return fail(DPF_EINVAL, "key column %d must be FOR or DELTA", key_col);
  ht.npay = B.n_payload;
  ht.dim_rows = kc.nrows;
  Q.build_key = kidx;
  Q.build_npay = B.n_payload;
  // Predicates in the given order, 32-bit ones first: a 64-bit range (a
  // FOR64 column) runs over survivors only, and when every predicate is one
  // a pass-all step that reads nothing leads (base = 1).
  std::vector<int> porder;
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < B.n_preds; ++i) {
      auto it = c->cols.find(B.preds[i].col);
      const bool wide = it != c->cols.end() && it->second.codec == C_FOR64;
      if (wide == (pass == 1)) porder.push_back(i);
    }
  bool all_wide = B.n_preds > 0;
  for (int i = 0; i < B.n_preds; ++i) {
    auto it = c->cols.find(B.preds[i].col);
    all_wide = all_wide && it != c->cols.end() && it->second.codec == C_FOR64;
  }
  const int base = all_wide ? 1 : 0;
  if (base + B.n_preds + B.n_joins > kMaxSteps) return fail(DPF_EINVAL, "build compiles to more than %d steps", kMaxSteps);
  double sel = 1.0;
  for (int k = 0; k < B.n_preds; ++k) {
    const dpf_pred& pr = B.preds[porder[size_t(k)]];
    int idx;
    if ((st = cs.add(pr.col, &idx))) return st;
    if ((st = compile_pred(c->cols[pr.col], pr, Q.steps[base + k], idx))) return st;
    sel *= std::min(1.0, step_selectivity(Q.steps[base + k], &c->cols[pr.col], nullptr));
  }
  if (base) {
    DevStep& A = Q.steps[0];
    std::memset(&A, 0, sizeof A);
    A.kind = ST_ALL;
    A.col = Q.steps[1].col;
    A.zlo = INT32_MIN;
    A.zhi = INT32_MAX;
  }
  std::vector<const HashTable*> probed;
  for (int j = 0; j < B.n_joins; ++j) {
    const dpf_join& J = B.joins[j];
    auto it = c->hts.find(J.ht);
    if (it == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", J.ht);
    if (it->second.failed) return fail(DPF_EINVAL, "hash table %d failed to build", J.ht);
    int idx;
    if ((st = cs.add(J.fk_col, &idx))) return st;
    const int codec = c->cols[J.fk_col].codec;
    if (codec != C_FOR && codec != C_DELTA) return fail(DPF_EINVAL, "join column %d must be FOR or DELTA", J.fk_col);
    const HashTable& H = it->second;
    DevStep& S = Q.steps[base + B.n_preds + j];
    std::memset(&S, 0, sizeof S);
    S.kind = ST_PROBE;
    S.col = uint8_t(idx);
    S.ht_kind = uint8_t(H.kind);
    if (H.kind == HT_DIRECT || H.kind == HT_RANK) {
      S.ht = H.kind == HT_DIRECT ? static_cast<const void*>(H.direct) : static_cast<const void*>(H.rank);
      S.kmin = H.kmin;
      S.krange = H.capacity;
    } else {
      S.ht = H.slots;
      S.ht_mask = H.capacity - 1;
    }
    S.zlo = H.key_lo;
    S.zhi = H.key_hi;
    sel *= std::min(1.0, step_selectivity(S, nullptr, &H));
    probed.push_back(&H);
  }
  for (int f = 0; f < B.n_payload; ++f) {
    const dpf_payload& F = B.payload[f];
    if (F.kind == DPF_PAYLOAD_COLUMN) {
      int idx;
      if ((st = cs.add(F.col, &idx))) return st;
      const Column& pc = c->cols[F.col];
      if (pc.codec != C_DICT) return fail(DPF_EINVAL, "payload column %d must be DICT", F.col);
      Q.build_pay[f] = idx;
      ht.pay_dom[f] = uint32_t(pc.dict.size());
      ht.pay_dict[f] = pc.d_dict;
    } else if (F.kind == DPF_PAYLOAD_JOIN) {
      if (F.join < 0 || F.join >= B.n_joins) return fail(DPF_EINVAL, "payload field %d names join %d", f, F.join);
      const HashTable& H = *probed[size_t(F.join)];
      if (F.field < 0 || F.field >= H.npay) return fail(DPF_EINVAL, "hash table %d has no payload field %d", H.id, F.field);
      // the build kernel decodes -1 - (2 * step + field)
      Q.build_pay[f] = -1 - (2 * (base + B.n_preds + F.join) + F.field);
      ht.pay_dom[f] = H.pay_dom[F.field];
      ht.pay_dict[f] = H.pay_dict[F.field];
    } else {
      return fail(DPF_EINVAL, "unknown payload kind %d", F.kind);
    }
  }
  Q.nsteps = uint32_t(base + B.n_preds + B.n_joins);
  // The payload fields through the survivor entries' group-id bits when
  // they fit there (the entries hold 32 - kRowBits bits of group id): a
  // probed table's field by its probe step's multiplier, a DICT column's
  // code by a key step after the filters.  The build kernel then reads each
  // kept row's fields from its entry instead of probing or decoding again.
  {
    uint32_t fbits[2] = {0, 0}, total = 0, keys = 0;
    for (int f = 0; f < B.n_payload; ++f) {
      while ((uint64_t(1) << fbits[f]) < uint64_t(std::max<uint32_t>(ht.pay_dom[f], 1u))) ++fbits[f];
      total += fbits[f];
      keys += B.payload[f].kind == DPF_PAYLOAD_COLUMN;
    }
    if (B.n_payload > 0 && total <= 20 && Q.nsteps + keys <= uint32_t(kMaxSteps)) {
      uint32_t shift = 0;
      for (int f = 0; f < B.n_payload; ++f) {
        const dpf_payload& F = B.payload[f];
        if (F.kind == DPF_PAYLOAD_COLUMN) {
          DevStep& K = Q.steps[Q.nsteps++];
          std::memset(&K, 0, sizeof K);
          K.kind = ST_KEY;
          K.col = uint8_t(Q.build_pay[f]);
          K.key_mul = 1u << shift;
          K.zlo = INT32_MIN;
          K.zhi = INT32_MAX;
        } else {
          DevStep& S = Q.steps[base + B.n_preds + F.join];
          (F.field == 0 ? S.mul0 : S.mul1) += 1u << shift;
        }
        Q.build_pay[f] = kPayFromGid | int32_t(shift << 8) | int32_t(fbits[f]);
        shift += fbits[f];
      }
    }
  }
  Q.nrows = cs.nrows;
  Q.page_rows = cs.page_rows;
  bs.host = cs.host;
  bs.wide_payload = B.n_payload == 2 && ht.pay_dom[0] == 65536 && ht.pay_dom[1] == 65536;
  bs.est_kept = double(kc.nrows) * sel;
  ht.table = kc.table;
  return DPF_OK;
}

// Chooses the layout of a table for at most `kept` rows whose keys lie in
// [lo, hi], allocates it and enqueues its initialisation on s: a direct
// table (one word per key of the range, one load per probe) for dense
// ranges; a rank directory (presence bits and a running count per 64 keys,
// then the payloads in key order: 2 bits per key of the range plus a word
// per row) for large ranges; open addressing (a power of two >= 2 x kept
// slots) otherwise.
static dpf_status alloc_table(dpf_ctx* c, const BuildSpec& bs, uint64_t kept, int64_t lo, int64_t hi, HashTable& ht,
                              BuildLaunch& L, cudaStream_t s) {
  const uint64_t range = kept && lo <= hi ? uint64_t(hi - lo + 1) : 0;
  if (range) {
    ht.key_lo = int32_t(lo);
    ht.key_hi = int32_t(hi);
  }
  dpf_status st;
  cudaError_t e;
  if (!bs.wide_payload && range > kDirectMaxRange && range <= kRankMaxRange) {
    const uint64_t nwords = (range + 63) / 64, nblocks = (nwords + 1023) / 1024;
    ht.kind = HT_RANK;
    ht.kmin = int32_t(lo);
    ht.capacity = uint32_t(range);
    const uint64_t bytes = 16 * nwords + 4 * kept;
    if (kept > UINT32_MAX) return fail(DPF_ENOMEM, "rank table of %llu rows is too large", (unsigned long long)kept);
    if ((st = dev_alloc(c, bytes + 4 * nblocks, reinterpret_cast<void**>(&ht.rank))) ||
        (st = dev_alloc(c, 16 + 8 * kept, reinterpret_cast<void**>(&ht.stage))))
      return st;
    L.rank_dir = reinterpret_cast<uint4*>(ht.rank);
    L.rank_pay = reinterpret_cast<uint32_t*>(ht.rank + 16 * nwords);
    L.rank_sums = reinterpret_cast<uint32_t*>(ht.rank + bytes);
    L.stage_n = reinterpret_cast<unsigned long long*>(ht.stage);
    L.rank_stage = reinterpret_cast<uint2*>(ht.stage + 16);
    L.rank_cap = uint32_t(kept);
    L.kmin = ht.kmin;
    L.krange = ht.capacity;
    e = cudaMemsetAsync(ht.rank, 0, 16 * nwords, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ht.stage, 0, 16, s);
  } else if (!bs.wide_payload && range <= std::max<uint64_t>(64 * kept, 1u << 20) && range <= kDirectMaxRange) {
    ht.kind = HT_DIRECT;
    ht.kmin = range ? int32_t(lo) : 0;
    ht.capacity = uint32_t(range);
    if ((st = dev_alloc_t(c, std::max<uint64_t>(range, 1), &ht.direct))) return st;
    L.direct = ht.direct;
    L.kmin = ht.kmin;
    L.krange = ht.capacity;
    e = launch_init_direct(ht.direct, uint32_t(std::max<uint64_t>(range, 1)), s);
  } else {
    uint64_t cap = 16;
    while (cap < 2 * kept) cap <<= 1;
    if (cap > (1ull << 31)) return fail(DPF_ENOMEM, "hash table of %llu entries is too large", (unsigned long long)kept);
    if ((st = dev_alloc_t(c, cap, &ht.slots))) return st;
    ht.kind = HT_OPEN;
    ht.capacity = uint32_t(cap);
    L.table = ht.slots;
    L.mask = uint32_t(cap - 1);
    e = launch_init_table(ht.slots, uint32_t(cap), s);
  }
  if (e != cudaSuccess) return fail(DPF_ECUDA, "hash table initialisation: %s", cudaGetErrorString(e));
  return DPF_OK;
}

static dpf_status build_status_error(uint32_t status, dpf_col_id key_col) {
  if (status & S_DUPKEY) return fail(DPF_EDUPKEY, "duplicate key in hash build of column %d", key_col);
  if (status & S_CORRUPT) return fail(DPF_EINVAL, "key column %d holds the reserved key INT32_MIN or corrupt data", key_col);
  return fail(DPF_EINTERNAL, "hash build status %u", status);
}

// Exact sizing: a count pass finds the kept rows and their key range, the
// host reads them back and sizes the table, then the insert pass fills it.
static dpf_status build_hash_impl(dpf_ctx* c, const dpf_build& B, void* stream, dpf_ht_id* out) {
  if (!c || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BuildSpec bs;
  dpf_status st = compile_build(c, B, bs);
  if (st) return st;
  HashTable& ht = bs.ht;
  DevQuery* dq;
  if ((st = dev_alloc_t(c, 1, &dq))) return st;
  BuildLaunch L{};
  L.q = dq;
  L.count = c->bcount;
  L.sched = c->bsched;
  L.nrows = bs.Q.nrows;
  L.page_rows = bs.Q.page_rows;
  L.host_data = bs.host;
  L.kminmax = c->bkminmax;
  unsigned long long kept = 0;
  int32_t minmax[2] = {INT32_MAX, INT32_MIN};
  uint32_t status = 0;
  auto cleanup = [&](dpf_status r) {
    dev_free(c, dq);
    return r;
  };
  cudaError_t e = cudaMemcpyAsync(dq, &bs.Q, sizeof bs.Q, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->bcount, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->bsched, 0, sizeof(Sched), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->bkminmax, minmax, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_build_count(L, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kept, c->bcount, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(minmax, c->bkminmax, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(fail(DPF_ECUDA, "hash build (count): %s", cudaGetErrorString(e)));
  if ((st = alloc_table(c, bs, kept, minmax[0], minmax[1], ht, L, s))) {
    free_table(c, ht);
    return cleanup(st);
  }
  ht.entries = kept;
  e = launch_build_insert(L, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &c->bsched->status, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || status) {
    free_table(c, ht);
    if (e != cudaSuccess) return cleanup(fail(DPF_ECUDA, "hash build (insert): %s", cudaGetErrorString(e)));
    return cleanup(build_status_error(status, B.key_col));
  }
  dev_free(c, ht.stage);  // the build has finished with it
  ht.stage = nullptr;
  ht.id = c->next_ht++;
  c->hts[ht.id] = ht;
  *out = ht.id;
  return cleanup(DPF_OK);
}

// Sizing from what is known at load time, so nothing is read back: the key
// column's bounds from its mini block headers and its row count as the
// bound on the kept rows.  Everything is enqueued on the stream; the
// table's device-side status and inserted-row count are read by
// finish_build once the stream has passed the build.
static dpf_status build_hash_async_impl(dpf_ctx* c, const dpf_build& B, void* stream, bool deferred,
                                        dpf_ht_id* out) {
  if (!c || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  // a deferred table is set up on the private stream and left empty
  cudaStream_t s = deferred ? c->io : static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return fail(DPF_EINVAL, "dpf_build_hash_async allocates and copies from host memory: it cannot be captured");
  }
  BuildSpec bs;
  dpf_status st = compile_build(c, B, bs);
  if (st) return st;
  HashTable& ht = bs.ht;
  const Column& kc = c->cols[B.key_col];
  BuildLaunch L{};
  if ((st = dev_alloc_t(c, 1, &ht.bq)) || (st = dev_alloc(c, sizeof(BuildStat), reinterpret_cast<void**>(&ht.bstat)))) {
    free_table(c, ht);
    return st;
  }
  L.q = ht.bq;
  L.sched = &ht.bstat->sched;
  L.inserted = &ht.bstat->inserted;
  L.nrows = bs.Q.nrows;
  L.page_rows = bs.Q.page_rows;
  L.host_data = bs.host;
  cudaError_t e = cudaMemcpyAsync(ht.bq, &bs.Q, sizeof bs.Q, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ht.bstat, 0, sizeof(BuildStat), s);
  if (e != cudaSuccess) {
    free_table(c, ht);
    return fail(DPF_ECUDA, "hash build: %s", cudaGetErrorString(e));
  }
  if ((st = alloc_table(c, bs, kc.nrows, kc.vmin, kc.vmax, ht, L, s))) {
    cudaStreamSynchronize(s);  // the copies above write blocks that free_table returns to the cache
    free_table(c, ht);
    return st;
  }
  e = cudaEventCreateWithFlags(&ht.done, cudaEventDisableTiming);
  if (!deferred) {
    if (e == cudaSuccess) e = launch_build_insert(L, s);
    if (e == cudaSuccess) e = cudaEventRecord(ht.done, s);
  } else if (e == cudaSuccess) {
    e = cudaHostAlloc(reinterpret_cast<void**>(&ht.hstat), sizeof(BuildStat), cudaHostAllocDefault);
    if (e == cudaSuccess) std::memset(ht.hstat, 0, sizeof(BuildStat));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // an empty table, scan uploaded, until a chain runs the build
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);  // nothing of the failed build may still be running when its blocks are freed
    free_table(c, ht);
    return fail(DPF_ECUDA, "hash build: %s", cudaGetErrorString(e));
  }
  ht.bl = L;
  ht.deferred = deferred;
  ht.pending = !deferred;
  ht.key_col = B.key_col;
  ht.entries = uint64_t(std::llround(bs.est_kept));  // an estimate until finish_build
  ht.id = c->next_ht++;
  c->hts[ht.id] = ht;
  *out = ht.id;
  return DPF_OK;
}

// Completes an asynchronous build: waits for it, reads its status and the
// rows it inserted, and releases its launch buffers.  A failed build keeps
// its error: the table stays allocated (plans already enqueued may read
// it) but no new plan or build may use it.
static dpf_status finish_build(dpf_ctx* c, HashTable& ht) {
  if (!ht.pending) return ht.failed ? fail(ht.failed, "hash table %d failed to build", ht.id) : DPF_OK;
  BuildStat bs{};
  cudaError_t e = cudaEventSynchronize(ht.done);
  if (e == cudaSuccess && ht.hstat) {
    bs = *ht.hstat;  // the launch copied it there before the event
  } else {
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bs, ht.bstat, sizeof bs, cudaMemcpyDeviceToHost, c->io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->io);
  }
  if (e != cudaSuccess) return fail(DPF_ECUDA, "hash build: %s", cudaGetErrorString(e));
  ht.pending = false;
  if (!ht.deferred) {  // a deferred table keeps its launch buffers for the next chain launch
    dev_free(c, ht.bq);
    dev_free(c, ht.bstat);
    dev_free(c, ht.stage);
    cudaEventDestroy(ht.done);
    ht.bq = nullptr;
    ht.bstat = nullptr;
    ht.stage = nullptr;
    ht.done = nullptr;
  }
  ht.entries = bs.inserted;
  if (bs.sched.status) {
    const dpf_status r = build_status_error(bs.sched.status, ht.key_col);
    ht.failed = r;
    return r;
  }
  return DPF_OK;
}

dpf_status dpf_build_hash(dpf_ctx* c, dpf_col_id key_col, const dpf_col_id* payload_cols, int32_t n_payload,
                          const dpf_pred* preds, int32_t n_preds, void* stream, dpf_ht_id* out) {
  if (n_payload < 0 || n_payload > 2 || (n_payload && !payload_cols)) return fail(DPF_EINVAL, "0..2 payload columns");
  dpf_payload pay[2] = {};
  for (int f = 0; f < n_payload; ++f) {
    pay[f].kind = DPF_PAYLOAD_COLUMN;
    pay[f].col = payload_cols[f];
  }
  dpf_build B{};
  B.key_col = key_col;
  B.n_payload = n_payload;
  B.payload = pay;
  B.n_preds = n_preds;
  B.preds = preds;
  return build_hash_impl(c, B, stream, out);
}

dpf_status dpf_build_hash_probe(dpf_ctx* c, const dpf_build* spec, void* stream, dpf_ht_id* out) {
  if (!spec) return fail(DPF_EINVAL, "NULL build description");
  return build_hash_impl(c, *spec, stream, out);
}

dpf_status dpf_build_hash_async(dpf_ctx* c, const dpf_build* spec, void* stream, dpf_ht_id* out) {
  if (!spec) return fail(DPF_EINVAL, "NULL build description");
  return build_hash_async_impl(c, *spec, stream, false, out);
}

dpf_status dpf_build_hash_deferred(dpf_ctx* c, const dpf_build* spec, dpf_ht_id* out) {
  if (!spec) return fail(DPF_EINVAL, "NULL build description");
  return build_hash_async_impl(c, *spec, nullptr, true, out);
}

dpf_status dpf_prepare_chain(dpf_ctx* c, const dpf_ht_id* builds, int32_t n_builds, const dpf_plan* plans,
                             int32_t n, const dpf_tuning* tuning, dpf_prep_id* out) {
  if (!c || !out || !builds) return fail(DPF_EINVAL, "NULL argument");
  if (n_builds < 1 || n_builds > 64) return fail(DPF_EINVAL, "need 1..64 deferred tables");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  std::vector<HashTable*> hs;
  for (int32_t i = 0; i < n_builds; ++i) {
    auto it = c->hts.find(builds[i]);
    if (it == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", builds[i]);
    if (!it->second.deferred) return fail(DPF_EINVAL, "hash table %d was not made by dpf_build_hash_deferred", builds[i]);
    if (it->second.failed) return fail(DPF_EINVAL, "hash table %d failed to build", builds[i]);
    if (std::find(hs.begin(), hs.end(), &it->second) != hs.end())
      return fail(DPF_EINVAL, "hash table %d is named twice", builds[i]);
    hs.push_back(&it->second);
  }
  Prep* p;
  dpf_status st = prepare(c, plans, n, tuning, &p);
  if (st) return st;
  p->chain = hs;
  for (HashTable* h : hs) ++h->refs;
  *out = p->id;
  return DPF_OK;
}

dpf_status dpf_hash_wait(dpf_ctx* c, dpf_ht_id id) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->hts.find(id);
  if (it == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", id);
  return finish_build(c, it->second);
}

dpf_status dpf_hash_info(dpf_ctx* c, dpf_ht_id id, uint64_t* entries, uint64_t* capacity) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->hts.find(id);
  if (it == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", id);
  if (dpf_status st = finish_build(c, it->second)) return st;
  if (entries) *entries = it->second.entries;
  if (capacity) *capacity = it->second.capacity;
  return DPF_OK;
}

dpf_status dpf_drop_hash(dpf_ctx* c, dpf_ht_id id) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->hts.find(id);
  if (it == c->hts.end()) return fail(DPF_EINVAL, "unknown hash table %d", id);
  if (it->second.refs > 0) return fail(DPF_EINVAL, "hash table %d is rebuilt by a prepared chain", id);
  cudaDeviceSynchronize();
  free_table(c, it->second);
  c->hts.erase(it);
  return DPF_OK;
}

dpf_status dpf_prepare(dpf_ctx* c, const dpf_plan* plans, int32_t n, const dpf_tuning* tuning, dpf_prep_id* out) {
  if (!c || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p;
  dpf_status st = prepare(c, plans, n, tuning, &p);
  if (st) return st;
  *out = p->id;
  return DPF_OK;
}

dpf_status dpf_context_device(dpf_ctx* c, int32_t* device) {
  if (!c || !device) return fail(DPF_EINVAL, "NULL argument");
  *device = c->device;
  return DPF_OK;
}

dpf_status dpf_autotune(dpf_ctx* c, const dpf_plan* plans, int32_t n, void* stream, uint32_t reps, dpf_tuning* best,
                        float* best_ms) {
  if (!c || !plans) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (reps == 0) reps = 3;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  static const uint32_t kChunk[] = {1024, 2048, 4096, 16384, 65536, 262144};
  static const uint32_t kThreads[] = {128, 256, 512, 1024};
  static const int32_t kPlace[] = {DPF_HT_AUTO, DPF_HT_SMEM, DPF_HT_GLOBAL};
  static const uint32_t kCtas[] = {0, uint32_t(kFusedMinBlocksHi)};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(DPF_ECUDA, "cudaEventCreate failed");
  }
  dpf_tuning top{};
  float top_ms = -1.f;
  dpf_status last = DPF_OK;
  // Times one configuration; keeps it when it is the fastest so far.
  // Returns a status only for errors that end the search.
  auto trial = [&](dpf_tuning t) -> dpf_status {
    Prep* p = nullptr;
    dpf_status st = prepare(c, plans, n, &t, &p);
    if (st) {  // e.g. the tables do not fit this configuration
      last = st;
      return DPF_OK;
    }
    const int32_t id = p->id;
    cudaError_t e = launch_prep(p, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) e = launch_prep(p, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    uint32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, &p->sched->status, 4, cudaMemcpyDeviceToHost);
    dpf_tuning used = p->tuning;
    release_prep(c, p);
    c->preps.erase(id);
    if (e != cudaSuccess) return fail(DPF_ECUDA, "autotune: %s", cudaGetErrorString(e));
    if (status) return fail(status & S_CORRUPT ? DPF_ECORRUPT : DPF_EINTERNAL, "autotune: device status %u", status);
    ms /= float(reps);
    if (top_ms < 0.f || ms < top_ms) {
      top_ms = ms;
      used.ctas_per_sm = t.ctas_per_sm;  // 0: the 3-CTA build at its occupancy; 4: the 4-CTA build
      top = used;
    }
    return DPF_OK;
  };
  dpf_status st = DPF_OK;
  // the launch grid (unstaged, one atomic per row)
  for (uint32_t cr : kChunk)
    for (uint32_t th : kThreads)
      for (int32_t pl : kPlace)
        for (uint32_t ct : kCtas) {
          if (st || (th > 256 && ct != 0)) continue;  // one build per wide CTA size
          dpf_tuning t{};
          t.chunk_rows = cr;
          t.threads = th;
          t.ht_placement = pl;
          t.ctas_per_sm = ct;
          t.staging = DPF_STAGE_OFF;
          t.group_agg = DPF_GROUP_AGG_ATOMIC;
          st = trial(t);
        }
  // then, at the fastest point, the staging ring and warp-aggregated group-by
  if (!st && top_ms >= 0.f) {
    dpf_tuning t = top;
    t.staging = DPF_STAGE_ON;
    if (t.threads > 256) t.threads = 256;  // the staging builds take 256-thread CTAs
    st = trial(t);
  }
  if (!st && top_ms >= 0.f) {
    dpf_tuning t = top;
    t.group_agg = DPF_GROUP_AGG_WARP;
    st = trial(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (top_ms < 0.f) return fail(last ? last : DPF_EINVAL, "autotune: no configuration could be prepared");
  c->tune_cache[plans_signature(c, plans, n)] = top;
  if (best) *best = top;
  if (best_ms) *best_ms = top_ms;
  return DPF_OK;
}

dpf_status dpf_plan_footprint(dpf_ctx* c, const dpf_plan* plan, uint64_t* bytes) {
  if (!c || !plan || !bytes) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DevQuery Q;
  bool host = false;
  std::vector<const HashTable*> probes;
  dpf_status st = compile_plan(c, *plan, Q, &host, probes);
  if (st) return st;
  const uint64_t S1 = 1 + Q.naggs;
  *bytes = align16(uint64_t(Q.domain) * S1 * 8) + 32 + align16(uint64_t(std::max<uint32_t>(Q.domain, 1)) * sizeof(dpf_record)) +
           sizeof(DevQuery) + 8;
  return DPF_OK;
}

dpf_status dpf_launch(dpf_ctx* c, dpf_prep_id id, void* stream) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, id);
  if (!p) return fail(DPF_EINVAL, "unknown batch %d", id);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(launch_prep(p, s));
  CUDA_TRY(cudaEventRecord(p->ev, s));
  p->launched = true;
  return DPF_OK;
}

dpf_status dpf_capture_graph(dpf_ctx* c, dpf_prep_id id, void* stream) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, id);
  if (!p) return fail(DPF_EINVAL, "unknown batch %d", id);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return fail(DPF_EINVAL, "graph capture needs a non-default stream");
  if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
  if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
  // set the smem attribute before capture (not a stream operation)
  fused_blocks_per_sm(p->L.threads, p->L.acc_slots, p->L.smem_tables, p->L.host_data, p->L.min_blocks,
                      p->L.stage_bw);
  CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_prep(p, s);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(DPF_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  p->graph = graph;
  CUDA_TRY(cudaGraphInstantiate(&p->gexec, graph, 0));
  return DPF_OK;
}

dpf_status dpf_launch_graph(dpf_ctx* c, dpf_prep_id id, void* stream) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, id);
  if (!p || !p->gexec) return fail(DPF_EINVAL, "batch %d has no captured graph", id);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaGraphLaunch(p->gexec, s));
  CUDA_TRY(cudaEventRecord(p->ev, s));
  for (HashTable* h : p->chain) h->pending = true;
  p->launched = true;
  return DPF_OK;
}

dpf_status dpf_read_result(dpf_ctx* c, dpf_prep_id id, int32_t i, dpf_record* buf, uint64_t cap, uint64_t* n_out,
                           int32_t timeout_ms) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, id);
  if (!p) return fail(DPF_EINVAL, "unknown batch %d", id);
  return read_result(c, p, i, buf, cap, n_out, timeout_ms);
}

dpf_status dpf_prepare_unfused(dpf_ctx* c, const dpf_plan* plan, dpf_prep_id* out) {
  if (!c || !plan || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  dpf_tuning t{};
  t.ht_placement = DPF_HT_GLOBAL;
  Prep* p;
  dpf_status st = prepare(c, plan, 1, &t, &p);
  if (st) return st;
  const DevQuery& Q = p->hq[0];
  if (p->L.host_data) {
    dpf_release(c, p->id);
    return fail(DPF_EINVAL, "the unfused chain reads device-resident columns only");
  }
  for (uint32_t k = 0; k < Q.nsteps; ++k)
    if (Q.steps[k].kind == ST_CONTAINS || Q.steps[k].kind == ST_LIKE || Q.cols[Q.steps[k].col].codec == C_FSST) {
      dpf_release(c, p->id);
      return fail(DPF_EINVAL, "the unfused chain evaluates PREFIX on STR columns only (no FSST, no CONTAINS)");
    }
  for (uint32_t i = 0; i < Q.ncols; ++i)
    if (Q.cols[i].codec == C_FOR64) {
      dpf_release(c, p->id);
      return fail(DPF_EINVAL, "the unfused chain decodes 32-bit columns only (no FOR64)");
    }
  const uint64_t n = Q.nrows;
  // layout: per column decoded arrays, flags, two (rid, gid) lists, counts
  uint64_t bytes = 0;
  std::vector<uint64_t> off_v(Q.ncols), off_l(Q.ncols), off_o(Q.ncols);
  uint64_t fixed = 0;
  for (uint32_t i = 0; i < Q.ncols; ++i) {
    if (Q.cols[i].codec == C_STR) {
      off_l[i] = bytes; bytes += align16(4 * n);
      off_o[i] = bytes; bytes += align16(8 * n);
      fixed += 12 * n;
    } else {
      off_v[i] = bytes; bytes += align16(4 * n);
      fixed += 4 * n;
    }
  }
  const uint64_t off_flags = bytes; bytes += align16(n);
  fixed += n;
  uint64_t off_list[4];
  for (int k = 0; k < 4; ++k) { off_list[k] = bytes; bytes += align16(4 * n); }
  const uint64_t off_counts = bytes; bytes += 8 * kUnfusedCounts;
  if ((st = dev_alloc(c, bytes, reinterpret_cast<void**>(&p->unf_scratch)))) {
    dpf_release(c, p->id);
    return st;
  }
  UnfusedChain& U = p->U;
  U.q = Q;
  U.dq = p->dq;
  for (uint32_t i = 0; i < Q.ncols; ++i) {
    if (Q.cols[i].codec == C_STR) {
      U.lens[i] = reinterpret_cast<int32_t*>(p->unf_scratch + off_l[i]);
      U.offs[i] = reinterpret_cast<uint64_t*>(p->unf_scratch + off_o[i]);
    } else {
      U.vals[i] = reinterpret_cast<int32_t*>(p->unf_scratch + off_v[i]);
    }
  }
  U.flags = p->unf_scratch + off_flags;
  U.rid[0] = reinterpret_cast<uint32_t*>(p->unf_scratch + off_list[0]);
  U.gid[0] = reinterpret_cast<uint32_t*>(p->unf_scratch + off_list[1]);
  U.rid[1] = reinterpret_cast<uint32_t*>(p->unf_scratch + off_list[2]);
  U.gid[1] = reinterpret_cast<uint32_t*>(p->unf_scratch + off_list[3]);
  U.counts = reinterpret_cast<unsigned long long*>(p->unf_scratch + off_counts);
  U.sched = p->sched;
  p->unfused = true;
  p->fixed_inter_bytes = fixed;
  *out = p->id;
  return DPF_OK;
}

dpf_status dpf_prep_stats(dpf_ctx* c, dpf_prep_id id, uint32_t* launches, uint64_t* inter) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, id);
  if (!p) return fail(DPF_EINVAL, "unknown batch %d", id);
  if (launches) *launches = p->launches;
  if (inter) {
    *inter = 0;
    if (p->unfused) {
      if (p->launched) {
        CUDA_TRY(cudaEventSynchronize(p->ev));
        unsigned long long counts[kUnfusedCounts];
        CUDA_TRY(cudaMemcpyAsync(counts, p->U.counts, sizeof counts, cudaMemcpyDeviceToHost, c->io));
        CUDA_TRY(cudaStreamSynchronize(c->io));
        uint64_t lists = 0;
        for (int k = 0; k < kUnfusedCounts; ++k) lists += counts[k] * 8;
        *inter = p->fixed_inter_bytes + lists;
      } else {
        *inter = p->fixed_inter_bytes;
      }
    }
  }
  return DPF_OK;
}

dpf_status dpf_parse_tuning(const char* json, dpf_tuning* out) {
  if (!out) return fail(DPF_EINVAL, "NULL argument");
  dpf_tuning t{};
  std::string why;
  if (json && *json && !parse_tuning_json(json, &t, &why)) return fail(DPF_EINVAL, "tuning: %s", why.c_str());
  *out = t;
  return DPF_OK;
}

dpf_status dpf_set_tuning(dpf_ctx* c, const char* json) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  dpf_tuning t{};
  if (dpf_status st = dpf_parse_tuning(json, &t)) return st;
  c->defaults = t;
  return DPF_OK;
}

dpf_status dpf_prep_tuning(dpf_ctx* c, dpf_prep_id id, dpf_tuning* out) {
  if (!c || !out) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  Prep* p = find_prep(c, id);
  if (!p) return fail(DPF_EINVAL, "unknown batch %d", id);
  *out = p->tuning;
  return DPF_OK;
}

dpf_status dpf_release(dpf_ctx* c, dpf_prep_id id) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  auto it = c->preps.find(id);
  if (it == c->preps.end()) return fail(DPF_EINVAL, "unknown batch %d", id);
  release_prep(c, it->second.get());
  c->preps.erase(it);
  return DPF_OK;
}

dpf_status dpf_execute_plan(dpf_ctx* c, const dpf_plan* plans, int32_t n, void* stream, dpf_query_id* out_ids) {
  if (!c || !out_ids) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p;
  dpf_status st = prepare(c, plans, n, nullptr, &p);
  if (st) return st;
  p->oneshot = true;
  st = dpf_launch(c, p->id, stream);
  if (st) {
    const std::string msg = t_last_error;
    dpf_release(c, p->id);
    return fail(st, "%s", msg.c_str());
  }
  for (int i = 0; i < n; ++i) out_ids[i] = (dpf_query_id(p->id) << 20) | i;
  return DPF_OK;
}

dpf_status dpf_fetch_result(dpf_ctx* c, dpf_query_id id, dpf_record* buf, uint64_t cap, uint64_t* n_out,
                            int32_t timeout_ms) {
  if (!c) return fail(DPF_EINVAL, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Prep* p = find_prep(c, dpf_prep_id(id >> 20));
  const int32_t i = int32_t(id & 0xfffff);
  if (!p || !p->oneshot || i >= p->nq || p->fetched[i]) return fail(DPF_ENOTFOUND, "unknown or fetched query id %lld", (long long)id);
  dpf_status st = read_result(c, p, i, buf, cap, n_out, timeout_ms);
  if (st) return st;
  p->fetched[i] = 1;
  if (std::all_of(p->fetched.begin(), p->fetched.end(), [](char f) { return f != 0; })) {
    const int32_t pid = p->id;
    release_prep(c, p);
    c->preps.erase(pid);
  }
  return DPF_OK;
}

}  // extern "C"

/*
 * dpf.h -- C ABI of the GB300 fused columnar query library.
 *
 * The library implements the data path of Data Path Fusion (arxiv 2605.10511):
 * compressed columnar pages are taken through decompression, predicates,
 * hash-join probes and hash aggregation inside ONE persistent GPU kernel per
 * query batch, without materialising intermediates in global memory and
 * without host intervention during execution (Sec. 3.1, Sec. 3.2).  The join
 * tables a plan probes are built by fused scan + build (Kernel #1) and scan +
 * probe + build (Kernel #2) kernels, so multi-table join chains run as one
 * pipeline per table.
 *
 * Conventions for every call:
 *   - Return value: 0 (DPF_OK) or a negative dpf_status.  No C++ exception
 *     crosses the ABI.  After an error, dpf_last_error() returns a message
 *     (thread-local, valid until the next call on the same thread).
 *   - Pointers named `host` are host memory, `device` are device memory;
 *     `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - The library never frees or retains caller memory: inputs are copied
 *     or consumed before the call returns (asynchronous calls copy what they
 *     need at call time).
 *   - A context is bound to one CUDA device.  Calls on one context are
 *     serialised by an internal mutex; objects are not shared across
 *     contexts.
 */
#ifndef DPF_H
#define DPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef int32_t dpf_status;
#define DPF_OK 0
#define DPF_EINVAL (-1)     /* bad argument, unknown id, type mismatch         */
#define DPF_ENOMEM (-2)     /* allocation failed or the memory budget is spent */
#define DPF_ECUDA (-3)      /* a CUDA runtime call failed                      */
#define DPF_EDUPKEY (-4)    /* duplicate key in a hash-table build             */
#define DPF_EBUSY (-5)      /* admission refused (serving)                     */
#define DPF_ETIMEOUT (-6)   /* result not ready within the timeout             */
#define DPF_ETRUNC (-7)     /* caller buffer too small; *n_out = needed count  */
#define DPF_ENOTFOUND (-8)  /* unknown or already fetched query id             */
#define DPF_ECORRUPT (-9)   /* a page or mini block header failed validation   */
#define DPF_EINTERNAL (-10) /* device-side invariant violated (bounded probe)  */

typedef struct dpf_ctx dpf_ctx;
typedef int32_t dpf_col_id;
typedef int32_t dpf_ht_id;
typedef int64_t dpf_query_id;
typedef int32_t dpf_prep_id;

/* Thread-local description of the last error on this thread. */
const char* dpf_last_error(void);

/* ----------------------------------------------------------- context */
/* Device-memory hooks (e.g. a framework's caching allocator).  alloc must
 * return 256-byte aligned device memory usable from any stream of the
 * context's device, or NULL on failure.  NULL hooks = cudaMalloc/cudaFree. */
typedef struct dpf_alloc_hooks {
  void* (*alloc)(uint64_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} dpf_alloc_hooks;

/* Creates a context on `device`.  hbm_budget caps the device bytes the
 * context may hold (0 = no cap); allocations beyond it fail with
 * DPF_ENOMEM (Sec. 4.3: the build side must fit in GPU memory). */
dpf_status dpf_create(dpf_ctx** out, int32_t device, uint64_t hbm_budget,
                      const dpf_alloc_hooks* hooks);
/* Waits for the context's work, frees every object it owns. */
dpf_status dpf_destroy(dpf_ctx* ctx);
/* Device bytes held by the context's live objects (columns, hash tables,
 * prepared batches).  Without allocation hooks, freed blocks of up to 64 MiB
 * (1 GiB in all) are kept for reuse and not counted here; with a budget, live
 * plus kept bytes stay within it.  dpf_destroy returns all of them. */
dpf_status dpf_memory_used(dpf_ctx* ctx, uint64_t* bytes);
/* CUDA device the context is bound to. */
dpf_status dpf_context_device(dpf_ctx* ctx, int32_t* device);

/* ----------------------------------------------------------- columns */
/* Storage encodings (Sec. 3.4, Sec. 4.1).  Every encoding splits a column
 * into pages of `page_rows` rows and pages into mini blocks of 128 values,
 * each mini block preceded by metadata {FOR base, bit width, offset}
 * (Sec. 3.4.1).  Page byte layout: see the storage-format section of the
 * repository's design notes; it is identical for host and device. */
enum dpf_codec {
  DPF_CODEC_FOR = 1,   /* int32: frame of reference + bit packing (GPU-FOR)          */
  DPF_CODEC_DELTA = 2, /* int32: deltas of consecutive rows, FOR-packed (sorted keys) */
  DPF_CODEC_DICT = 3,  /* int32 with <= 65536 distinct values: sorted dictionary,
                          FOR-packed ranks (Sec. 3.4.1, short CHAR as integers)       */
  DPF_CODEC_STR = 4,   /* bytes: FOR-packed lengths + per-mini-block start + raw bytes
                          (Sec. 3.4.2 variable-length page)                           */
  DPF_CODEC_FSST = 5,  /* bytes: FSST-encoded strings (Sec. 3.4.2, Sec. 4.1) in the STR
                          page layout.  A column table of <= 255 symbols of 1..8 bytes;
                          code c < nsym stands for symbol c, code 255 for the literal
                          byte that follows.  The table travels in the dict arrays as
                          nsym int32 triples {bytes 0..3, bytes 4..7, length}         */
  DPF_CODEC_FOR64 = 6  /* int64 (BIGINT): 64-bit GPU-FOR (Sec. 4.1): per mini block an
                          int64 base, a bit width 0..64 and 2*bw packed 64-bit words,
                          field j at bit j*bw (a field may cross into the next word).
                          A plan reads FOR64 columns as aggregate operands (int64,
                          wrapping) and in predicates (int64 compares; see dpf_op);
                          joins and group keys take 32-bit columns                  */
};
/* Where a column's pages live: device HBM, or pinned host memory read by
 * the kernel directly through the host link (oversize tables). */
enum dpf_placement { DPF_PLACE_DEVICE = 0, DPF_PLACE_HOST_PINNED = 1 };

typedef struct dpf_column_desc {
  int32_t codec;      /* enum dpf_codec                                           */
  int32_t placement;  /* enum dpf_placement                                       */
  uint32_t page_rows; /* rows per page: multiple of 128 in [128, 2^20]; 0 = 65536 */
  int32_t table;      /* caller's table id: columns scanned together by one plan
                         must share table, row count and page_rows                */
} dpf_column_desc;

/* Host-side encoder (the data loader of Sec. 4.2), no device work.
 *   values: host int32[nrows] (FOR/DELTA/DICT), int64[nrows] (FOR64) or
 *           host bytes (STR/FSST)
 *   str_offsets: host uint64[nrows+1] byte offsets into values (STR/FSST
 *                only, str_offsets[0] may be non-zero), else NULL
 *   out: host buffer of `cap` bytes for the page images, or NULL to size
 *   page_off: host uint64[npages+1] (npages = ceil(nrows/page_rows)), filled
 *   row_prefix: host uint64[npages] RID index (cumulative rows, Sec. 3.4.2)
 *   dict/dict_cap/dict_n: DICT: sorted distinct values; FSST: the symbol
 *                table as 3 int32 per symbol (<= 765); may be NULL to size,
 *                *dict_n receives the int32 count
 *   size_out: receives the encoded byte size
 * Errors: DPF_EINVAL (nrows = 0, bad codec/page_rows, > 65536 distinct for
 * DICT, a page too large for the format), DPF_ETRUNC (cap or dict_cap too
 * small; *size_out / *dict_n hold the needed sizes). */
dpf_status dpf_encode_column(const dpf_column_desc* desc, const void* values,
                             const uint64_t* str_offsets, uint64_t nrows, uint8_t* out,
                             uint64_t cap, uint64_t* page_off, uint64_t* row_prefix,
                             int32_t* dict, uint64_t dict_cap, uint64_t* dict_n,
                             uint64_t* size_out);

/* Uploads already encoded pages (host memory, layout as produced by
 * dpf_encode_column) to the column's placement; validates every page header.
 * Errors: DPF_EINVAL, DPF_ECORRUPT (bad page), DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_load_encoded(dpf_ctx* ctx, const dpf_column_desc* desc, const uint8_t* pages,
                            uint64_t size, const uint64_t* page_off, const uint64_t* row_prefix,
                            uint64_t nrows, const int32_t* dict, uint64_t dict_n,
                            dpf_col_id* out);

/* Encodes on the host (dpf_encode_column) and uploads (dpf_load_encoded).
 * The caller keeps ownership of `values` / `str_offsets`. */
dpf_status dpf_load_column(dpf_ctx* ctx, const dpf_column_desc* desc, const void* values,
                           const uint64_t* str_offsets, uint64_t nrows, dpf_col_id* out);

/* Rows, encoded bytes (page images) and raw bytes (4/row, 8/row for FOR64,
 * or string bytes + 8/row of offsets) of a loaded column; any out pointer
 * may be NULL. */
dpf_status dpf_column_info(dpf_ctx* ctx, dpf_col_id col, uint64_t* rows,
                           uint64_t* encoded_bytes, uint64_t* raw_bytes);

/* Copies `bytes` of a column's page images starting at byte `offset` back
 * to host memory (inspection and tests). */
dpf_status dpf_column_read(dpf_ctx* ctx, dpf_col_id col, uint64_t offset, uint64_t bytes,
                           uint8_t* host_out);

dpf_status dpf_drop_column(dpf_ctx* ctx, dpf_col_id col);

/* --------------------------------------------------------- predicates */
/* On a FOR64 (BIGINT) column the comparisons, BETWEEN and IN with one
 * operand compare the int64 value with the int64 operands (other ops:
 * DPF_EINVAL).  Such a predicate runs over the rows that pass the other
 * steps; when every filter of a scan is one, every row is decoded for it. */
enum dpf_op {
  DPF_OP_LT = 0, DPF_OP_LE = 1, DPF_OP_GT = 2, DPF_OP_GE = 3, DPF_OP_EQ = 4,
  DPF_OP_NE = 5,
  DPF_OP_BETWEEN = 6, /* v[0] <= x <= v[1], both ends inclusive                 */
  DPF_OP_IN = 7,      /* x in {v[0..n)}, 1 <= n <= DPF_MAX_IN                     */
  DPF_OP_PREFIX = 8,  /* STR/FSST: string starts with prefix[0..prefix_len); a
                         prefix longer than the string does not match; an empty
                         prefix matches every row (Sec. 4.1 variable-length scan) */
  DPF_OP_CONTAINS = 9,/* STR/FSST: prefix[0..prefix_len) occurs anywhere in the
                         string (LIKE '%pattern%'; Sec. 4.1 names KMP matching);
                         an empty pattern matches every row                       */
  DPF_OP_LIKE = 10    /* SQL LIKE: the whole string against prefix[0..prefix_len)
                         where '%' stands for any run of bytes and '_' for any
                         one byte (no escape character).  'p%' and '%p%' with a
                         wildcard-free p run as PREFIX / CONTAINS (STR or FSST);
                         other patterns need a STR column                        */
};
#define DPF_MAX_IN 8
#define DPF_MAX_PREFIX 32

typedef struct dpf_pred {
  dpf_col_id col;          /* column of the scanned table                          */
  int32_t op;              /* enum dpf_op                                          */
  int32_t n;               /* IN: number of operands                               */
  int32_t prefix_len;      /* PREFIX / CONTAINS: 0..DPF_MAX_PREFIX                 */
  int64_t v[DPF_MAX_IN];   /* operands, compared with the int32 value as int64;
                              for DICT columns they are dictionary values          */
  uint8_t prefix[DPF_MAX_PREFIX];
} dpf_pred;

/* --------------------------------------------------------- hash tables */
/* Kernel #1 of Sec. 3.1: scans a dimension table's key column and payload
 * columns, keeps the rows passing every predicate (conjunction) and inserts
 * key -> payload into an open-addressing hash table in device memory.
 *   key_col: FOR or DELTA column; keys must be unique among the rows kept
 *            and differ from INT32_MIN
 *   payload_cols: 0..2 DICT columns of the same table; field f of a probe hit
 *            is the dictionary code of payload_cols[f]
 * Asynchronous on `stream` except for one device-to-host read of the kept
 * row count (the table is sized from it).  Errors: DPF_EINVAL,
 * DPF_EDUPKEY, DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_build_hash(dpf_ctx* ctx, dpf_col_id key_col, const dpf_col_id* payload_cols,
                          int32_t n_payload, const dpf_pred* preds, int32_t n_preds,
                          void* stream, dpf_ht_id* out);
/* Entries and slot capacity of a built table (waits for an asynchronous
 * build, see dpf_build_hash_async, and returns its error if it failed). */
dpf_status dpf_hash_info(dpf_ctx* ctx, dpf_ht_id ht, uint64_t* entries, uint64_t* capacity);
dpf_status dpf_drop_hash(dpf_ctx* ctx, dpf_ht_id ht);

/* ---------------------------------------------------------------- plans */
/* One pipeline ending in hash aggregation (Kernel #3 of Sec. 3.1):
 *   SELECT keys, COUNT(*), aggs FROM fact JOIN dims WHERE preds GROUP BY keys
 * All fact columns named by a plan belong to one table.  Aggregates are
 * int64 over sign-extended int32 inputs (Sec. 4.3), wrapping on overflow. */
typedef struct dpf_join {
  dpf_col_id fk_col; /* column of the scanned table probed (FOR or DELTA) */
  dpf_ht_id ht;      /* table built by dpf_build_hash or dpf_build_hash_probe */
} dpf_join;

/* ------------------------------------------------ scan, probe and build */
/* Kernel #2 of Sec. 3.1: scans a table, probes tables built earlier and
 * inserts the rows that pass into a new table, which a later pipeline
 * probes.  A row is kept when it passes every predicate AND finds a match
 * in every join (inner joins, probed through columns of the scanned table).
 * A chain such as LINEITEM -> ORDERS -> CUSTOMER is built table by table:
 * CUSTOMER with dpf_build_hash, then ORDERS with this call probing the
 * CUSTOMER table, then the fused plan over LINEITEM probes the ORDERS table.
 * Payload field f of the new table is either the dictionary code of a DICT
 * column of the scanned table, or payload field `field` of the row's match
 * in joins[join] (carried through the chain, so a plan over LINEITEM can
 * group by a CUSTOMER attribute).  Keys, limits, errors and synchronisation
 * are those of dpf_build_hash; at most DPF_MAX_JOINS joins and
 * DPF_MAX_PREDS predicates. */
enum dpf_payload_kind { DPF_PAYLOAD_COLUMN = 0, DPF_PAYLOAD_JOIN = 1 };
typedef struct dpf_payload {
  int32_t kind;      /* enum dpf_payload_kind                                 */
  dpf_col_id col;    /* DPF_PAYLOAD_COLUMN: DICT column of the scanned table  */
  int32_t join;      /* DPF_PAYLOAD_JOIN: index into dpf_build.joins          */
  int32_t field;     /* DPF_PAYLOAD_JOIN: payload field of that join's table  */
} dpf_payload;
typedef struct dpf_build {
  dpf_col_id key_col;                           /* FOR or DELTA             */
  int32_t n_payload; const dpf_payload* payload; /* 0..2                    */
  int32_t n_preds;   const dpf_pred* preds;     /* conjunction              */
  int32_t n_joins;   const dpf_join* joins;     /* inner joins              */
} dpf_build;
dpf_status dpf_build_hash_probe(dpf_ctx* ctx, const dpf_build* spec, void* stream, dpf_ht_id* out);

/* Kernels #1 / #2 of Sec. 3.1 without any device-to-host read, so a chain's
 * builds and the plan that probes the last table can be enqueued back to
 * back on one stream (the paper launches its three kernels in sequence).
 * The same scan as dpf_build_hash_probe (spec->n_joins may be 0), but the
 * table is sized from what is known at load time: the key column's value
 * bounds from its mini block headers and its row count as the bound on
 * the rows kept.  Such a table can be larger than an exactly sized one
 * (open addressing: 2 x the scanned rows; a rank directory: one payload
 * word per scanned row).
 *   stream: every kernel and copy of the build is enqueued on it, and the
 *           call returns once they are; the table is ready when the stream
 *           reaches that point, so plans and builds that probe it must run
 *           on the same stream (or wait on an event recorded after it).
 *           It cannot be captured into a CUDA graph (DPF_EINVAL): the call
 *           allocates the table and copies its compiled scan from host
 *           memory.
 * Errors that only the kernels can find (a duplicate key: DPF_EDUPKEY; the
 * reserved key INT32_MIN: DPF_EINVAL) are reported by dpf_hash_wait or
 * dpf_hash_info, which wait for the build; a table whose build failed
 * stays allocated (plans already enqueued may read it; every access stays
 * within it) and is refused by later dpf_prepare and build calls.  Until
 * then dpf_prepare uses an estimate of its entry count for step ordering.
 * Errors at the call: DPF_EINVAL, DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_build_hash_async(dpf_ctx* ctx, const dpf_build* spec, void* stream, dpf_ht_id* out);
/* Waits for a table's build (returns at once for tables built by the
 * synchronous calls) and reports its outcome: DPF_OK, DPF_EDUPKEY,
 * DPF_EINVAL (the reserved key or corrupt pages), DPF_EINTERNAL or
 * DPF_ECUDA.  The same error is returned again by later calls. */
dpf_status dpf_hash_wait(dpf_ctx* ctx, dpf_ht_id ht);

/* Kernel #1 / #2 of Sec. 3.1 prepared but not run: the scan is compiled
 * and uploaded and the table allocated, sized as dpf_build_hash_async
 * sizes it, and left empty (every probe misses) until a chain prepared by
 * dpf_prepare_chain runs the build.  The call waits for its own set-up on
 * the library's private stream and enqueues nothing on the caller's.
 * Errors: DPF_EINVAL, DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_build_hash_deferred(dpf_ctx* ctx, const dpf_build* spec, dpf_ht_id* out);

enum dpf_key_kind { DPF_KEY_COLUMN = 0, DPF_KEY_PAYLOAD = 1 };
typedef struct dpf_key {
  int32_t kind;      /* DPF_KEY_COLUMN: fact DICT column `col`;
                        DPF_KEY_PAYLOAD: field `field` of join `join`      */
  dpf_col_id col;
  int32_t join;
  int32_t field;
} dpf_key;

enum dpf_agg_op {
  DPF_AGG_COUNT = 0,   /* COUNT(*)              */
  DPF_AGG_SUM = 1,     /* SUM(int64 a)          */
  DPF_AGG_SUM_MUL = 2, /* SUM(int64 a * b)      */
  DPF_AGG_SUM_SUB = 3  /* SUM(int64 a - b)      */
};
typedef struct dpf_agg {
  int32_t op;
  dpf_col_id a, b;     /* FOR/DELTA columns of the fact table (b unused for SUM) */
} dpf_agg;

#define DPF_MAX_PREDS 8
#define DPF_MAX_JOINS 4
#define DPF_MAX_KEYS 2
#define DPF_MAX_AGGS 4
#define DPF_MAX_GROUPS 65536  /* product of the key dictionary sizes */

typedef struct dpf_plan {
  int32_t n_preds;  const dpf_pred* preds;  /* on fact columns, conjunction */
  int32_t n_joins;  const dpf_join* joins;  /* inner equi-joins, in order   */
  int32_t n_keys;   const dpf_key* keys;    /* group keys, <= 2             */
  int32_t n_aggs;   const dpf_agg* aggs;    /* <= 4                         */
  dpf_col_id scan_col; /* any column of the scanned table; names the table
                          when no predicate, join, key or aggregate does
                          (e.g. a bare COUNT(*)); 0 = none              */
} dpf_plan;

/* Launch configuration; 0 in a field = chosen by the library (tuning cache,
 * then defaults). */
/* Join-table placement (Sec. 4.3 keeps the build side in GPU memory; where
 * in it is ours): AUTO = the table of the first (dense) step in shared memory
 * when it fits 48 KB, the tables of later steps in device memory; SMEM = every
 * table that fits the opt-in shared memory, in probe order; GLOBAL = every
 * table in device memory (served by L1/L2). */
enum dpf_ht_place { DPF_HT_AUTO = 0, DPF_HT_SMEM = 1, DPF_HT_GLOBAL = 2 };
typedef struct dpf_tuning {
  uint32_t chunk_rows;   /* rows per scheduling ticket (one warp's unit of work):
                            multiple of 512, at most 2^24; default 4096        */
  uint32_t threads;      /* threads per CTA: 128 or 256; 512 or 1024 (2 / 1 CTAs
                            per SM) for device-resident, unstaged batches
                            without CONTAINS / FSST steps                    */
  int32_t ht_placement;  /* enum dpf_ht_place                                     */
  uint32_t ctas_per_sm;  /* persistent CTAs per SM: 0 = as many as fit of the
                            kernel build for 3 resident 256-thread CTAs
                            (80 registers); >= 4 = the build for 4 (64
                            registers) when four fit, else as for 0          */
  int32_t staging;       /* enum dpf_staging: copy the first (dense) step's
                            compressed mini blocks into a per-warp shared-
                            memory ring with asynchronous copies a tile ahead
                            of their decode (Sec. 3.2 IO stage overlapped with
                            decompression); integer first steps over device-
                            resident pages only                              */
  int32_t group_agg;     /* enum dpf_group_agg: how grouped aggregates are added
                            into the accumulators: one int64 atomic per row,
                            or warp-aggregated (lanes of a round holding the
                            same group, found by __match_any_sync, add once) */
} dpf_tuning;
enum dpf_staging { DPF_STAGE_DEFAULT = 0, DPF_STAGE_ON = 1, DPF_STAGE_OFF = 2 };
enum dpf_group_agg { DPF_GROUP_AGG_DEFAULT = 0, DPF_GROUP_AGG_WARP = 1, DPF_GROUP_AGG_ATOMIC = 2 };
/* The context's default launch configuration: the fields a dpf_prepare
 * leaves 0 (or a NULL tuning) and dpf_autotune has not chosen for its
 * plans take these before the library's defaults.  json is a flat JSON
 * object with any of the keys of dpf_tuning: "chunk_rows", "threads",
 * "ctas_per_sm" (non-negative integers, as dpf_tuning constrains them),
 * "ht_placement" ("auto" | "smem" | "global"), "staging" ("default" | "on"
 * | "off"), "group_agg" ("default" | "warp" | "atomic"); the enums may also
 * be given by their values.  NULL or "" resets to the library's defaults.
 * Errors: DPF_EINVAL (a syntax error, an unknown key, a bad value; the
 * previous defaults stay). */
dpf_status dpf_set_tuning(dpf_ctx* ctx, const char* json);
/* The parse of dpf_set_tuning alone (no context, no device): json (NULL or
 * "" gives all zeros) into *out.  Errors: DPF_EINVAL. */
dpf_status dpf_parse_tuning(const char* json, dpf_tuning* out);

/* Result record: keys are dictionary values (0 when unused); count = rows
 * in the group; val[i] = aggregate i (COUNT repeats count). */
typedef struct dpf_record {
  int32_t key[2];
  int64_t count;
  int64_t val[4];
} dpf_record;

/* Prepares a batch of n plans for repeated launches: validates them,
 * compiles them to the device plan format, allocates accumulators and
 * result buffers.  Errors: DPF_EINVAL (type mismatch, unknown id, a group
 * domain above DPF_MAX_GROUPS), DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_prepare(dpf_ctx* ctx, const dpf_plan* plans, int32_t n, const dpf_tuning* tuning,
                       dpf_prep_id* out);
/* A join chain as one prepared batch (Sec. 3.1: Kernels #1 / #2 build the
 * tables, Kernel #3 probes them): every launch of the batch (dpf_launch,
 * or a graph captured by dpf_capture_graph and replayed by
 * dpf_launch_graph) first rebuilds the deferred tables builds[0..n_builds)
 * in that order (each emptied, then scanned, probing the tables built
 * before it), then runs the plans, all on one stream with no host work in
 * between.  Inner tables come first.  A launch's build status and entry
 * counts are read by dpf_hash_wait(builds[i]) after it; a failed build is
 * sticky (later dpf_prepare and build calls refuse the table).  The
 * tables stay referenced while the batch exists: dpf_drop_hash refuses
 * them until dpf_release.  Two batches rebuilding the same table must not
 * run at the same time.  Tune (dpf_autotune) after a launch has filled
 * the tables.  Errors: DPF_EINVAL (unknown, non-deferred, failed or
 * repeated table; the errors of dpf_prepare), DPF_ENOMEM, DPF_ECUDA. */
dpf_status dpf_prepare_chain(dpf_ctx* ctx, const dpf_ht_id* builds, int32_t n_builds,
                             const dpf_plan* plans, int32_t n_plans, const dpf_tuning* tuning,
                             dpf_prep_id* out);
/* Enqueues ONE persistent fused kernel for all plans of the batch on
 * `stream` (no host synchronisation, capturable into a CUDA graph).  The
 * kernel leaves its scratch state zeroed, so launches can be replayed. */
dpf_status dpf_launch(dpf_ctx* ctx, dpf_prep_id prep, void* stream);
/* Captures dpf_launch into a CUDA graph owned by the prepared batch;
 * dpf_launch_graph replays it on `stream`. */
dpf_status dpf_capture_graph(dpf_ctx* ctx, dpf_prep_id prep, void* stream);
dpf_status dpf_launch_graph(dpf_ctx* ctx, dpf_prep_id prep, void* stream);
/* Waits (up to timeout_ms; < 0 = forever) for the last launch of `prep`
 * and copies query i's records, ascending by key tuple, to host `buf`.
 * DPF_ETRUNC if cap < needed (*n_out = needed).  Device status words turn
 * into DPF_ECORRUPT / DPF_EINTERNAL. */
dpf_status dpf_read_result(dpf_ctx* ctx, dpf_prep_id prep, int32_t i, dpf_record* buf,
                           uint64_t cap, uint64_t* n_out, int32_t timeout_ms);
/* Tuning the batch will launch with (after defaults and cache lookup;
 * staging = DPF_STAGE_ON only when the batch is staged, group_agg =
 * DPF_GROUP_AGG_WARP only when some grouped query uses it). */
dpf_status dpf_prep_tuning(dpf_ctx* ctx, dpf_prep_id prep, dpf_tuning* out);
dpf_status dpf_release(dpf_ctx* ctx, dpf_prep_id prep);

/* Autotuner for batched launches.  Sec. 3.2 splits a table into chunks that
 * thread blocks process in a loop; the chunk size, the threads per block and
 * where the join tables live (shared memory vs device memory, Sec. 4.3) are
 * the launch configuration.  dpf_autotune prepares the n plans under each
 * configuration of a fixed grid (chunk_rows 1K..256K, threads 128..1024,
 * tables AUTO/SMEM/GLOBAL, kernel build for 3 or 4 CTAs per SM), then, at the
 * fastest point, staging on and warp-aggregated group-by; it times `reps`
 * launches of each on `stream` with CUDA
 * events after one warm-up launch (reps 0 = 3), and keeps the fastest in the
 * context's tuning cache under the plans' signature (the rows and encodings
 * of the columns they read, their steps, tables, groups and aggregates; not
 * predicate constants).  Later dpf_prepare calls on plans with the same
 * signature take the cached values for tuning fields left 0.  `best` and
 * `best_ms` (mean time per launch) may be NULL.  Runs the device work
 * synchronously.  Errors: as dpf_prepare; DPF_ECORRUPT / DPF_EINTERNAL from
 * the device status word. */
dpf_status dpf_autotune(dpf_ctx* ctx, const dpf_plan* plans, int32_t n, void* stream, uint32_t reps,
                        dpf_tuning* best, float* best_ms);
/* Device bytes one plan occupies while it runs (int64 accumulators of its
 * group domain, result records, device plan), for admission by memory
 * footprint.  Errors: as dpf_prepare. */
dpf_status dpf_plan_footprint(dpf_ctx* ctx, const dpf_plan* plan, uint64_t* bytes);

/* The unfused baseline: the same single plan prepared as a chain of one
 * kernel per operator that materialises every intermediate in device
 * memory (decoded columns, predicate flags, row-id lists after each join),
 * like the separate-kernel data path the paper compares with (Sec. 5.1).
 * Launched, captured and read with the calls above.  Errors as
 * dpf_prepare. */
dpf_status dpf_prepare_unfused(dpf_ctx* ctx, const dpf_plan* plan, dpf_prep_id* out);
/* Kernel launches per run and device bytes of intermediates written by the
 * last completed run (0 for the fused kernel); waits for that run. */
dpf_status dpf_prep_stats(dpf_ctx* ctx, dpf_prep_id prep, uint32_t* launches,
                          uint64_t* intermediate_bytes);

/* For callers that cannot allocate device memory while they run a query
 * (a framework that has reserved all device memory in its own pool, a
 * serving loop whose policy forbids allocation, code running inside another
 * allocator).  The paper has no counterpart; this is a library convenience.
 * Runs ONE plan through the fused kernel on `stream` and allocates nothing:
 * the kernel's scratch (scheduler counters, the compiled plan, the per-group
 * int64 accumulators) lives in a fixed region of DPF_NOALLOC_SCRATCH_BYTES
 * (1 MiB) of device memory that is part of the library image (every GPU
 * that loads the library holds it until the process exits).  The caller
 * passes the outputs:
 *   out: device dpf_record[cap], cap >= the plan's group domain (1 when
 *        ungrouped); records are written ascending by key tuple
 *   out_count: device uint32, receives the number of records
 * Asynchronous; read the outputs after synchronising `stream`.  The first
 * call on a device looks up the region's device address (a one-time set-up
 * per device).  The call copies its compiled plan from host memory that
 * lives only for the call, so it cannot be captured into a CUDA graph: on
 * a capturing stream it returns DPF_EINVAL and enqueues nothing.  Every
 * call shares the one region per device and clears it before use, so calls
 * whose kernels overlap on the GPU (different streams, or different
 * threads) race and give wrong results: serialise them.  Device-side data
 * checks are read back with dpf_noalloc_status.  Errors: DPF_EINVAL (a plan
 * needing more scratch than the region holds: DPF_NOALLOC_FIXED_BYTES +
 * 8 x domain x (1 + aggregates) bytes; cap below the domain; a capturing
 * stream; the dpf_prepare plan errors), DPF_ECUDA. */
#define DPF_NOALLOC_SCRATCH_BYTES (1u << 20)
#define DPF_NOALLOC_FIXED_BYTES 3328u /* scheduler state + compiled plan */
dpf_status dpf_execute_noalloc(dpf_ctx* ctx, const dpf_plan* plan, void* stream, dpf_record* out,
                               uint64_t cap, uint32_t* out_count);
/* Device status word of the last dpf_execute_noalloc kernel on the
 * context's device, read after the caller has synchronised that call's
 * stream (a blocking 4-byte copy; allocates nothing).  *bits = the raw word
 * (0 = clean).  Returns DPF_OK when clean, DPF_ECORRUPT when the kernel met
 * data that passed load validation but not its own checks (e.g. a
 * dictionary code beyond its dictionary: such rows are dropped), or
 * DPF_EINTERNAL (a bounded probe ran out of slots). */
dpf_status dpf_noalloc_status(dpf_ctx* ctx, uint32_t* bits);

/* Measurement aid (not part of the paper's method): the read bandwidth, in
 * GB/s (10^9 bytes/s), that a kernel on the context's device sees on a
 * buffer of `bytes` in device memory (DPF_PLACE_DEVICE) or in mapped pinned
 * host memory (DPF_PLACE_HOST_PINNED), read with 16-byte read-only loads by
 * every SM as the fused kernel reads pages; mean of `reps` passes (0 = 5)
 * after one warm-up pass, timed with CUDA events on `stream`.  The call
 * allocates and frees the buffer itself and waits for its work.  For
 * host-resident tables this is the roofline denominator of the fused
 * kernel's host-resident variant.  Errors: DPF_EINVAL (bytes not a multiple
 * of 16 in [1 MiB, 64 GiB], bad placement), DPF_ECUDA. */
dpf_status dpf_read_rate(dpf_ctx* ctx, int32_t placement, uint64_t bytes, uint32_t reps, void* stream,
                         double* gb_per_s);

/* One-shot form (Sec. 3.1): prepare + launch on `stream`; out_ids[i]
 * names plan i's result.  n > 1 runs every plan in one persistent launch. */
dpf_status dpf_execute_plan(dpf_ctx* ctx, const dpf_plan* plans, int32_t n, void* stream,
                            dpf_query_id* out_ids);
/* Blocks up to timeout_ms for a query of dpf_execute_plan and copies its
 * records (the "record format returned to the host" of Sec. 3.1).  On
 * DPF_ETRUNC nothing is consumed; on success the id is freed. */
dpf_status dpf_fetch_result(dpf_ctx* ctx, dpf_query_id id, dpf_record* buf, uint64_t cap,
                            uint64_t* n_out, int32_t timeout_ms);

/* ---------------------------------------------------------------- serving
 * A request loop over one context (not in the paper; the serving pattern
 * built on its batched fused launch).  Join tables and compressed columns
 * stay resident in the context; queries are submitted as plans over them.
 * A dispatcher thread owned by the server keeps up to max_inflight batches
 * on the device, each on its own stream, and launches the queued queries
 * (FIFO, up to max_batch per launch) as soon as a slot is free and their
 * device footprint (dpf_plan_footprint) fits mem_budget next to the
 * queries already running: continuous batching.  A query's records do not
 * depend on the batch it ran in. */
typedef struct dpf_server dpf_server;
typedef struct dpf_server_config {
  uint32_t max_batch;    /* plans per launch; 0 = 64, at most 4096                */
  uint32_t max_inflight; /* batches on the device at once; 0 = 2, at most 64      */
  uint64_t mem_budget;   /* device bytes of admitted queries at once; 0 = no cap  */
  dpf_tuning tuning;     /* launch configuration; 0 fields = cache / defaults     */
} dpf_server_config;
/* Host steady-clock times in microseconds since dpf_server_create. */
typedef struct dpf_query_times {
  double submit_us;    /* dpf_server_submit accepted the query              */
  double launch_us;    /* its batch was handed to the GPU                   */
  double done_us;      /* the dispatcher saw the batch complete             */
  uint32_t batch_size; /* queries in that launch                            */
} dpf_query_times;
typedef struct dpf_server_stats {
  uint64_t submitted, completed, failed, batches, launched_batches;
  uint64_t queued;       /* waiting for a slot or memory                    */
  uint64_t in_use_bytes; /* footprint of the queries on the device          */
} dpf_server_stats;
/* Starts the dispatcher thread.  cfg may be NULL (all defaults).  Errors:
 * DPF_EINVAL, DPF_ECUDA. */
dpf_status dpf_server_create(dpf_ctx* ctx, const dpf_server_config* cfg, dpf_server** out);
/* Queues one plan (copied at call time; validated with dpf_plan_footprint)
 * and returns its ticket.  DPF_EBUSY: its footprint alone exceeds
 * mem_budget, or the server is stopping. */
dpf_status dpf_server_submit(dpf_server* srv, const dpf_plan* plan, uint64_t* ticket);
/* Waits up to timeout_ms (< 0 = forever) for a ticket and copies its
 * records to host `buf`.  DPF_ETRUNC if cap < needed (*n_out = needed;
 * nothing consumed).  On success, and on a query error (returned as its
 * status), the ticket is collected.  `times` may be NULL. */
dpf_status dpf_server_wait(dpf_server* srv, uint64_t ticket, dpf_record* buf, uint64_t cap,
                           uint64_t* n_out, int32_t timeout_ms, dpf_query_times* times);
dpf_status dpf_server_stats_get(dpf_server* srv, dpf_server_stats* out);
/* Runs the queued and in-flight queries to completion, stops the
 * dispatcher and frees the server (results not collected are dropped). */
dpf_status dpf_server_destroy(dpf_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* DPF_H */

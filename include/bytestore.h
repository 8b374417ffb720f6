/*
 * bytestore.h -- C ABI of the GB300 ByteStore library (libbytestore.so).
 *
 * ByteStore (Zhang, Feng, Lo, Qin, "ByteStore: Hybrid Layouts for Main-Memory
 * Column Stores") stores each int32 column in one of three layouts and runs two
 * operations on it:
 *   - scan:   column + predicate -> result bit vector       (Section 2.2, Alg. 3)
 *   - lookup: column + result bit vector -> int32 values     (Section 2.2, Alg. 4)
 * Layouts: PP-VBS (prefix-preserving encoding, Algorithm 1, stored as Variable
 * Byte Slice, Section 3.2), ByteSlice (Section 2.5) and Bit-Packed (Section 2.3).
 *
 * Conventions shared by every entry point:
 *   - Return value: BS_OK (0) or a negative BS_ERR_* status. Nothing aborts.
 *   - Pointers named d_* are device pointers (CUDA global memory on the
 *     column's device); h_* are host pointers. The caller owns every buffer it
 *     passes; a bs_column owns its own device and host buffers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Scans and lookups are asynchronous and stream-ordered; a device-
 *     side consistency failure is recorded in a device status word and reported
 *     by bs_last_device_error() after the stream has been synchronised.
 *   - Result bit vectors are arrays of uint32 words: bit i of word w is row
 *     32*w + i (Section 3.3.1 builds R from 32-bit movemask words). A scan
 *     writes ceil(n/32) words and leaves every bit at or past n zero; input bit
 *     vectors may hold anything at or past n (it is ignored).
 *   - Literals are plain int32 values; the library encodes them with the
 *     column's dictionary (Section 2.2). Literals absent from the dictionary are
 *     rewritten to an equivalent predicate on present values.
 *   - Row ids are uint32 (a column has fewer than 2^32 rows).
 */
#ifndef BYTESTORE_H
#define BYTESTORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define BS_OK 0
#define BS_ERR_INVALID_ARG (-1)   /* bad pointer, size, op or layout */
#define BS_ERR_OOM (-2)           /* host or device allocation failed */
#define BS_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define BS_ERR_CAPACITY (-4)      /* output buffer smaller than the result */
#define BS_ERR_UNSUPPORTED (-5)   /* valid request this column cannot serve */
#define BS_ERR_TIMEOUT (-6)       /* a bounded device or host wait expired */
#define BS_ERR_DEVICE_CHECK (-7)  /* a kernel's bounds check fired */
#define BS_ERR_NOT_READY (-8)     /* asynchronous result not complete yet */

typedef enum { BS_BITPACKED = 0, BS_BYTESLICE = 1, BS_PPVBS = 2 } bs_layout;

/* Predicate types of Section 2.2; BETWEEN is inclusive on both ends. */
typedef enum { BS_LT = 0, BS_LE = 1, BS_GT = 2, BS_GE = 3, BS_EQ = 4, BS_NE = 5, BS_BETWEEN = 6 } bs_op;

typedef struct bs_column bs_column; /* opaque; owns its device buffers */

/* Encoding options (NULL selects all defaults).
 *   domain_bits / domain_min: for BS_BYTESLICE and BS_BITPACKED, declare the
 *       code of value v to be v - domain_min over [0, 2^domain_bits)
 *       (1 <= domain_bits <= 32). 0 = use a dictionary instead.
 *   domain_values / n_domain: for BS_BYTESLICE and BS_BITPACKED, a declared
 *       dictionary (distinct int32 values in any order); code = rank of the
 *       value in it. NULL = the column's observed distinct values. PP-VBS
 *       encodes the observed values with their frequencies (Algorithm 1)
 *       unless domain_counts is also given.
 *   domain_counts: with domain_values, for BS_PPVBS: the frequency of each
 *       declared value (same order, n_domain entries) that Algorithm 1 builds
 *       the codes from, instead of the column's own counts. A row shard of a
 *       larger column passes the whole column's dictionary and counts, so
 *       every shard gets the same codes and the shards' results concatenate
 *       to the whole column's. Every value of the column must be declared
 *       (else INVALID_ARG); declared values must be distinct.
 *   device: CUDA device ordinal, -1 = the current device.
 *   host_only: 1 = build the layout in host memory only (no GPU needed); such a
 *       column answers bs_column_row_codes / bs_column_get_info but not scans.
 *   keep_host: 1 = keep the host copy of the layout after the upload.
 *   threads: host encoder threads, 0 = every available core.
 *   categorical: for BS_PPVBS, 1 = codes by Algorithm 2 (categorical columns:
 *       most frequent values first, ties by smaller value; a balanced tree
 *       whose codes do not follow value order). Such a column answers only
 *       = and != (other predicates: UNSUPPORTED); lookups are unchanged. */
typedef struct {
    int32_t domain_bits;
    int32_t device;
    int64_t domain_min;
    const int32_t *domain_values;
    uint64_t n_domain;
    int32_t host_only;
    int32_t keep_host;
    int32_t threads;
    int32_t categorical;
    const uint64_t *domain_counts;
} bs_encode_opts;

/* ------------------------------------------------------------- columns */

/* Encode n int32 values (host memory, read only during the call) into `layout`
 * and upload the layout to the device (Section 2.2 dictionary encoding; PP-VBS
 * codes by Algorithm 1 and stored as VBS, Section 3.2; ByteSlice by Section 2.5;
 * Bit-Packed by Section 2.3). On success *out owns a new column; free it with
 * bs_column_free. n may be 0. Errors: INVALID_ARG (NULL pointers, n >= 2^32,
 * value outside a declared domain), OOM, CUDA. */
int bs_encode_column(const int32_t *h_values, uint64_t n, bs_layout layout,
                     const bs_encode_opts *opts, bs_column **out);

/* Write an encoded column to a file (the dictionary side and the layout's byte
 * arrays; a column without a host copy is read back from the device), so that
 * a column encoded once can be loaded instead of re-encoded. Errors:
 * INVALID_ARG (NULL, file not writable), UNSUPPORTED (neither a host nor a
 * device copy), CUDA. Not part of the paper. */
int bs_column_save(const bs_column *col, const char *path);

/* Read a column written by bs_column_save and place it like bs_encode_column
 * would (opts: device, host_only, keep_host; the other fields are ignored).
 * The file is checked for the magic, for sizes that fit the column's row
 * count and for the array sizes the kernels rely on. On success *out owns a
 * new column. Errors: INVALID_ARG (missing, truncated or inconsistent file),
 * OOM, CUDA. */
int bs_column_load(const char *path, const bs_encode_opts *opts, bs_column **out);

/* Test hook: build a column straight from codes, without a dictionary.
 * PP-VBS: h_codes[i] is an unpadded code of h_lens[i] bytes (1..8; first byte
 * most significant) -- any code set whose every extension of a shorter code has
 * a positive tail (the premise of Lemma 1). ByteSlice / Bit-Packed: h_codes[i]
 * < 2^code_bits, h_lens ignored (may be NULL). Such a column is scanned with
 * bs_scan_code and read back with bs_lookup_codes. */
int bs_column_from_codes(const uint64_t *h_codes, const uint8_t *h_lens, uint64_t n, bs_layout layout,
                         int32_t code_bits, const bs_encode_opts *opts, bs_column **out);

void bs_column_free(bs_column *col);

typedef struct {
    uint64_t n_rows;
    int32_t layout;          /* bs_layout */
    int32_t max_code_bytes;  /* PP-VBS: K (longest code); ByteSlice: number of slices */
    int32_t code_bits;       /* ByteSlice / Bit-Packed: k */
    int32_t on_device;
    uint64_t n_dict;         /* dictionary entries (0 for a declared range or raw codes) */
    uint64_t device_bytes;   /* HBM held by the column (layout + GPU index + decode tables) */
    uint64_t layout_bytes;   /* bytes of the paper's layout alone (Section 6.1.4 counts masks) */
    uint64_t len_hist[9];    /* PP-VBS: rows whose code has 1..8 bytes at [1..8] */
} bs_column_info;

int bs_column_get_info(const bs_column *col, bs_column_info *info);

/* Per-row codes (unpadded, first byte most significant) and lengths in bytes for
 * rows [row_begin, row_begin + count), read from the host copy of the layout.
 * ByteSlice / Bit-Packed report the k-bit code and length ceil(k/8).
 * Errors: INVALID_ARG (range), UNSUPPORTED (no host copy kept). */
int bs_column_row_codes(const bs_column *col, uint64_t row_begin, uint64_t count,
                        uint64_t *h_codes, uint8_t *h_lens);

/* The dictionary: sorted distinct values with their codes and code lengths
 * (PP-VBS: Algorithm 1's C and L; ByteSlice / Bit-Packed: the rank and ceil(k/8)).
 * Writes min(cap, n_dict) entries; any output may be NULL. */
int bs_column_dictionary(const bs_column *col, int32_t *h_values, uint64_t *h_codes, uint8_t *h_lens,
                         uint64_t cap);

/* --------------------------------------------------------------- scan */

/* Scan (Section 2.2; PP-VBS by Algorithm 3 and Lemma 1; ByteSlice and
 * Bit-Packed by Sections 2.5 and 2.3): bit i of d_bits = (v_i op lit), or
 * lit <= v_i <= lit2 for BS_BETWEEN (lit2 ignored otherwise). d_bits: device,
 * ceil(n/32) words, fully written. Errors: INVALID_ARG, UNSUPPORTED (raw-code
 * column or host-only column), CUDA. */
int bs_scan(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, uint32_t *d_bits, void *stream);

/* Seeded scan, the bit-vector pipelining of Section 3.3.1: d_bits = d_seed AND
 * scan(op, lit, lit2). Rows whose seed bit is 0 are never examined, so blocks
 * with an all-zero seed word stop before reading any byte slice. d_seed may
 * equal d_bits (in place). */
int bs_scan_seeded(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *d_seed,
                   uint32_t *d_bits, void *stream);

/* Scan with literal codes instead of values (raw-code columns and tests).
 * PP-VBS: code/len is an unpadded code of len bytes (1..8) compared with every
 * row's code as if both were zero-padded (Section 3.1.1). ByteSlice /
 * Bit-Packed: code is a k-bit code, len ignored. code2/len2: upper literal of
 * BS_BETWEEN. */
int bs_scan_code(const bs_column *col, bs_op op, uint64_t code, int32_t len, uint64_t code2, int32_t len2,
                 const uint32_t *d_seed, uint32_t *d_bits, void *stream);

/* One predicate of a conjunction. */
typedef struct {
    const bs_column *col;
    int32_t op;   /* bs_op */
    int32_t lit;
    int32_t lit2;
    int32_t reserved;
} bs_pred;

/* Conjunction of npreds (1..16) predicates over columns of equal length, each
 * scan seeded with the running result (Section 3.3.1, pipelined bit vectors).
 * d_bits: ceil(n/32) words. */
int bs_scan_conj(const bs_pred *preds, int32_t npreds, uint32_t *d_bits, void *stream);

/* ------------------------------------------------------------- lookup */

/* Device workspace bytes bs_lookup / bs_lookup_codes need for this column. */
uint64_t bs_lookup_workspace_bytes(const bs_column *col);

/* Lookup (Section 2.2, Algorithm 4): for every set bit i < n of d_bits, in
 * ascending row order, write v_i to d_out (device int32, out_cap entries).
 * The number of set bits is written to *d_count (device uint64, may be NULL)
 * even when it exceeds out_cap; only the first out_cap values are written.
 * d_workspace: device scratch of bs_lookup_workspace_bytes(col) bytes, or NULL
 * to let the call allocate (stream-ordered) and free it. */
int bs_lookup(const bs_column *col, const uint32_t *d_bits, int32_t *d_out, uint64_t out_cap,
              uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, void *stream);

/* Allocation-free lookup. The paper has no counterpart. It is for callers
 * that may not allocate device memory at the moment they look up: a process
 * that was granted a fixed device-memory budget up front and must not grow
 * it, a latency-critical path that must never wait on an allocator, or code
 * running where another component owns all allocation. Same arguments and
 * results as bs_lookup, but the scratch is a 2 MiB + 4 KiB array the library
 * keeps in device memory (held by every GPU that loads the library until the
 * process exits); the call makes no cudaMalloc, cudaFree or other allocating
 * call. Columns needing more scratch than that (2^32 rows or more; in
 * practice none, since n < 2^32) are rejected with BS_ERR_CAPACITY. The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and it keeps the previous call's contents;
 * nothing is cleared: the lookup's count kernel overwrites every scratch word
 * the later kernels of the same call read. Calls that overlap on the GPU, from
 * any stream or thread, race on the array and must be serialised by the
 * caller. */
int bs_lookup_noalloc(const bs_column *col, const uint32_t *d_bits, int32_t *d_out, uint64_t out_cap,
                      uint64_t *d_count, void *stream);

/* Same as bs_lookup but returns the zero-padded codes Algorithm 4 builds
 * (PP-VBS: K bytes; ByteSlice / Bit-Packed: the k-bit code) as uint64. */
int bs_lookup_codes(const bs_column *col, const uint32_t *d_bits, uint64_t *d_codes, uint64_t out_cap,
                    uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, void *stream);

/* ------------------------------------------------- fused scan + lookup */

/* Device workspace bytes bs_scan_lookup needs for a projection column of this
 * length (8 bytes per 4096 rows plus 256). */
uint64_t bs_scan_lookup_workspace_bytes(const bs_column *proj);

/* Fused scan + lookup (Section 2.2's query shape: a conjunction of predicates
 * evaluated by pipelined bit vectors, Section 3.3.1, then the lookup of a
 * projected column, Algorithm 4) in one kernel: the values of `proj` at the
 * rows where every predicate holds, in ascending row order, written to d_out
 * (device int32, out_cap entries; only the first out_cap values are written),
 * and the number of such rows to *d_count (device uint64, may be NULL) even
 * when it exceeds out_cap. The same results as bs_scan_conj followed by
 * bs_lookup, without the bit vector's round trip through memory and without
 * the lookup's separate count and offset kernels: each pair of tiles finds
 * its output offset from the counts of the earlier ones (decoupled look-back).
 * preds: 1..BS_MAX_CONJ predicates over columns of proj's length on proj's
 * device; proj NULL = preds[0].col. d_bits: NULL, or ceil(n/32) device words
 * that also receive the result bit vector (bits >= n zero). d_workspace:
 * device scratch of bs_scan_lookup_workspace_bytes(proj) bytes (cleared by
 * the call, stream-ordered), or NULL to let the call allocate and free it.
 * Errors: INVALID_ARG, UNSUPPORTED (raw-code or host-only columns, categorical
 * columns with an order predicate), CAPACITY (workspace too small), OOM, CUDA;
 * a look-back that gives up records BS_ERR_TIMEOUT for bs_last_device_error. */
int bs_scan_lookup(const bs_pred *preds, int32_t npreds, const bs_column *proj, uint32_t *d_bits, int32_t *d_out,
                   uint64_t out_cap, uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, void *stream);

/* Launch shape of bs_lookup's gather kernel for this column on its device
 * (introspection for tests and tuning): *parts = warps sharing one chunk of
 * 16 tiles (1, 2, 4, 8 or 16; short columns split chunks so that the resident
 * warps get about two units each), *grid = CTAs launched, *resident_ctas =
 * CTAs of that kernel resident on the whole GPU. Any pointer may be NULL. */
int bs_lookup_shape(const bs_column *col, int32_t *parts, int32_t *grid, int32_t *resident_ctas);

/* Lookup by row ids in caller order: d_out[t] = v_{d_rowids[t]}, t < m.
 * Row ids >= n set the device status word (BS_ERR_DEVICE_CHECK) and write 0. */
int bs_lookup_rowids(const bs_column *col, const uint32_t *d_rowids, uint64_t m, int32_t *d_out,
                     void *stream);

/* ------------------------------------------------ effective-bytes counter */

/* Bytes one scan must move at the kernels' granularity (32-byte sectors,
 * 256-row mask groups, 1024-row tiles), replayed on the host: the dense slice
 * sectors of lanes with rows to scan, then -- only for rows still equal to the
 * literal (early stop, Section 2.5 and Lemma 1) -- the M_j sectors of their
 * groups, the off_j entries and the BS_j sectors of the bytes compared (PP-VBS)
 * or the next slice's sectors (ByteSlice); Bit-Packed reads its whole stream.
 * paper_model_bytes is Algorithm 3 as printed (every mask word of levels
 * 2..min(l+1,K) loaded eagerly, 32-byte slice loads). Needs the host copy of
 * the layout (keep_host or host_only). h_seed: optional seed bit vector (host). */
typedef struct {
    uint64_t bytes;              /* dense + mask + offset + deep + result */
    uint64_t dense_bytes;
    uint64_t mask_bytes;
    uint64_t offset_bytes;
    uint64_t deep_bytes;
    uint64_t result_bytes;       /* result words written (+ seed words read) */
    uint64_t paper_model_bytes;
    uint64_t pending_rows[9];    /* rows still undecided entering byte j */
    uint64_t sampled_tiles;
} bs_scan_bytes_t;

int bs_scan_bytes(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_seed,
                  bs_scan_bytes_t *out);

/* bs_scan_bytes replaying every tile_stride-th tile only and scaling the
 * counts up by the tiles skipped (sampled_tiles says how many were replayed);
 * tile_stride = 1 is bs_scan_bytes. */
int bs_scan_bytes_sampled(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_seed,
                          uint64_t tile_stride, bs_scan_bytes_t *out);

/* Bytes one lookup must move: the bit vector once, 4 bytes per output value and
 * the distinct sectors of every gathered byte, mask group and offset entry
 * (decode tables are assumed cache-resident). h_bits: host bit vector. */
typedef struct {
    uint64_t bytes;
    uint64_t selected;
    uint64_t bits_bytes;
    uint64_t out_bytes;
    uint64_t dense_bytes;
    uint64_t mask_bytes;
    uint64_t offset_bytes;
    uint64_t deep_bytes;
} bs_lookup_bytes_t;

int bs_lookup_bytes(const bs_column *col, const uint32_t *h_bits, bs_lookup_bytes_t *out);

/* Bytes the fused scan + lookup (bs_scan_lookup) must move for one predicate
 * projected onto its own column: the scan's sectors as bs_scan_bytes counts
 * them, plus, for every row selected (h_sel: the predicate's result bit
 * vector, host memory), the sectors of the rest of its code with the M_j
 * sector and off_j entry of each level it reaches; each sector counted once.
 * result_bytes = 4 bytes per selected row (the values written) plus the bit
 * vector when write_bits != 0. Needs the host copy of the layout. PP-VBS and
 * Bit-Packed columns (a Bit-Packed scan already reads every code); ByteSlice:
 * BS_ERR_UNSUPPORTED. */
int bs_scan_lookup_bytes(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_sel,
                         int32_t write_bits, bs_scan_bytes_t *out);

/* ---------------------------------------------------- layout advisor */

#define BS_ADVISE_TIMED 0        /* Algorithm 5: time 100 scans per layout on the GPU */
#define BS_ADVISE_BYTES_MODEL 1  /* deterministic: bytes the scans must read, no timing */

typedef struct {
    int32_t layout;          /* chosen bs_layout (BS_BYTESLICE or BS_PPVBS) */
    int32_t n_points;        /* literals profiled (100) */
    double auc_byteslice;    /* area under the (selectivity, cost) curve */
    double auc_ppvbs;
    double selectivity[100];
    double cost_byteslice[100];  /* seconds (TIMED) or bytes (BYTES_MODEL) */
    double cost_ppvbs[100];
} bs_advice;

/* Column-layout advisor (Algorithm 5) for one column: encode it as ByteSlice
 * and as PP-VBS, profile `<` scans (numerical column) or `=` scans
 * (opts->categorical: PP-VBS by Algorithm 2) with 100 literals spread over the
 * selectivity range, integrate each profile by the trapezoid rule and keep the
 * smaller area (ties -> ByteSlice). opts as for bs_encode_column. */
int bs_advise_layout(const int32_t *h_values, uint64_t n, int32_t mode, const bs_encode_opts *opts,
                     bs_advice *out);

/* bs_advise_layout for predicates whose selectivity is known to lie in
 * [sel_lo, sel_hi] (0 <= sel_lo <= sel_hi <= 1; Section 5 notes the advisor
 * can take a known range into account): the 100 profiling literals are spread
 * over that range only. bs_advise_layout is the range [0, 1]. Errors as for
 * bs_advise_layout, INVALID_ARG for a bad range. */
int bs_advise_layout_range(const int32_t *h_values, uint64_t n, int32_t mode, const bs_encode_opts *opts,
                           double sel_lo, double sel_hi, bs_advice *out);

/* ------------------------------------------------------- batched form */

#define BS_MAX_CONJ 4

/* One request of a batch: a conjunction of 1..BS_MAX_CONJ predicates over
 * columns of equal length (pipelined bit vectors, Section 3.3.1), then the
 * lookup (Section 2.2, Algorithm 4) of the selected rows of `proj`. */
typedef struct {
    int32_t npreds;
    int32_t reserved;
    bs_pred preds[BS_MAX_CONJ];
    const bs_column *proj;  /* column looked up (same length); NULL = preds[0].col */
    int32_t *d_out;         /* device int32[out_cap]: values in ascending row order */
    uint64_t out_cap;
    uint64_t *d_count;      /* device uint64: number of selected rows (may exceed out_cap); may be NULL */
    uint32_t *d_bits;       /* optional device bit vector (ceil(n/32) words) receiving the scan
                               result; NULL = batch-owned scratch */
} bs_request;

/* Shape of the batched launch (NULL = defaults; any shape field set makes the
 * shape explicit: the unset ones take their defaults, no cache is read).
 *   threads: 128, 256 or 512 threads per CTA; 0 = the tuned (or default 256) shape.
 *   blocks_per_sm: CTAs per SM, 0 = as many as fit (all CTAs are co-resident).
 *   autotune: 1 = time candidate shapes on this batch and keep the fastest:
 *             threads x CTAs per SM, then around the best the ring stages,
 *             the chunks per claim and the early-stop granularity; the choice
 *             is cached per batch signature in tune_cache.
 *   use_graph: 1 (default) = capture the launch in a CUDA graph, 0 = launch directly.
 *   tune_cache: JSON-lines cache file, NULL = $BS_TUNE_CACHE (or no cache).
 *   stages: slices of the first predicate in flight per warp (2, 3 or 4; 0 = 3).
 *   unit_chunks: chunks of 16 tiles (16,384 rows) a warp takes per claim, i.e.
 *             rows per unit of work (1, 2 or 4; 0 = 1).
 *   stop_rows: early-stop granularity, the rows whose pending state decides
 *             whether a deeper level is read: 256 (one PP-VBS mask group, or
 *             the lanes of a ByteSlice tile that have pending rows) or 1024
 *             (the whole tile once any row is pending); 0 = 256. */
typedef struct {
    int32_t threads;
    int32_t blocks_per_sm;
    int32_t autotune;
    int32_t use_graph;
    const char *tune_cache;
    int32_t stages;
    int32_t unit_chunks;
    int32_t stop_rows;
    int32_t reserved;
} bs_batch_opts;

/* The shape a batch runs with. */
typedef struct {
    int32_t threads, blocks_per_sm, ctas, stages, unit_chunks, stop_rows, graph;
    int32_t persistent_requests;     /* requests run by the persistent kernel */
    int32_t single_query_requests;   /* requests run by the single-query kernels (columns of 2^28+ rows) */
} bs_batch_shape;

typedef struct bs_batch bs_batch; /* opaque: descriptors, scratch, captured graph */

/* Prepare a batch of nreq requests (1..65536) for repeated launches: encodes
 * every literal, uploads the request descriptors, allocates the batch scratch
 * (bit vectors not supplied by the caller, per-chunk counts and offsets) and
 * captures one CUDA graph: requests over columns of 2^28 rows or more run the
 * single-query scan and lookup kernels (as bs_scan_conj + bs_lookup would),
 * all others one persistent cooperative kernel. All columns must live on the
 * same device and outlive the batch; so must the caller's output buffers.
 * Errors: INVALID_ARG, UNSUPPORTED (raw-code column), OOM, CUDA. Not part of
 * the paper: its batched launch has no counterpart there. */
int bs_batch_create(const bs_request *reqs, int32_t nreq, const bs_batch_opts *opts, bs_batch **out);

/* Run every request of the batch with one launch (one graph launch, or one
 * cooperative kernel launch), stream-ordered. */
int bs_batch_launch(bs_batch *b, void *stream);

/* The shape the batch runs with: threads per CTA, CTAs, graph captured (0/1). */
int bs_batch_info(const bs_batch *b, int32_t *threads, int32_t *ctas, int32_t *graph);

/* The full launch shape of a batch (including the tuned parameters). */
int bs_batch_get_shape(const bs_batch *b, bs_batch_shape *out);

void bs_batch_free(bs_batch *b);

/* ------------------------------------------------------------- serving */

/* Upper bound of the rows a predicate selects, from the dictionary counts
 * (exact for PP-VBS and for dictionary-coded ByteSlice / Bit-Packed columns;
 * the row count for columns coded by a declared value range). */
int bs_estimate_rows(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, uint64_t *out);

/* A query for the server: a conjunction of 1..BS_MAX_CONJ predicates over
 * equal-length resident columns, then the lookup of `proj` (NULL = the first
 * predicate's column). */
typedef struct {
    int32_t npreds;
    int32_t reserved;
    bs_pred preds[BS_MAX_CONJ];
    const bs_column *proj;
} bs_query;

/* Server options (NULL or 0 fields = defaults).
 *   max_batch: queries per launch (64); slots: batches in flight on separate
 *   streams (2); result_bytes: device memory for result buffers, the admission
 *   cap (1 GiB); scratch_bytes: device memory for the bit vectors and chunk
 *   offsets of queries in flight (4 GiB); threads: batch kernel CTA size (256);
 *   device: CUDA device, -1 = current; single_query_kernels: 1 = every query
 *   runs the single-query scan and lookup kernels, never the persistent kernel
 *   (with max_batch = 1 and slots = 1 this is serial plain execution through
 *   the same dispatcher and admission). */
typedef struct {
    int32_t max_batch;
    int32_t slots;
    uint64_t result_bytes;
    uint64_t scratch_bytes;
    int32_t threads;
    int32_t device;
    int32_t single_query_kernels;
    int32_t reserved;
} bs_server_opts;

typedef struct {
    int32_t status;           /* BS_ERR_NOT_READY while queued or running; when done BS_OK, or why the
                               * query failed: BS_ERR_CUDA (its batch could not be launched),
                               * BS_ERR_DEVICE_CHECK (a bounds check failed in its batch's kernels),
                               * BS_ERR_TIMEOUT (a bounded device wait gave up); a failed query has
                               * count 0 and d_values NULL */
    int32_t reserved;
    uint64_t count;           /* selected rows */
    const int32_t *d_values;  /* device values, ascending row order; valid until bs_server_release */
    double queue_us;          /* submission -> launch */
    double latency_us;        /* submission -> results complete on the device (event observed) */
} bs_query_result;

typedef struct {
    uint64_t submitted, completed, rejected, batches;
    double mean_batch;
    uint64_t result_bytes_in_use, scratch_bytes_in_use;
    uint64_t queued;
    uint64_t failed;          /* completed queries whose status is not BS_OK */
    uint64_t persistent_queries;    /* queries run by the persistent kernel */
    uint64_t single_query_queries;  /* queries run by the single-query kernels */
} bs_server_stats;

typedef struct bs_server bs_server; /* opaque */

/* A serving loop over resident columns (the paper has no counterpart). A
 * dispatcher thread admits queued queries in arrival order while their result
 * buffers (bound from bs_estimate_rows) and scratch fit the budgets, packs the
 * admitted ones into a batch and launches it on a free slot's stream as
 * bs_batch_create's graph would run it (queries over columns of 2^28 rows or
 * more by the single-query kernels, the others by the persistent kernel, sized
 * to share the GPU with the other slots); queries arriving meanwhile join the
 * next batch (continuous batching). Columns must outlive the queries that use
 * them. Results stay in device memory until released. */
int bs_server_create(const bs_server_opts *opts, bs_server **out);

/* Enqueue a query (non-blocking). Errors: INVALID_ARG, UNSUPPORTED, CAPACITY
 * (the query can never fit the server's memory budgets). */
int bs_server_submit(bs_server *s, const bs_query *q, uint64_t *ticket);

/* Result of a ticket: BS_ERR_NOT_READY until it completes, then the query's
 * own status (also in res->status): BS_OK or the error that failed it. */
int bs_server_poll(bs_server *s, uint64_t ticket, bs_query_result *res);

/* Wait at most timeout_ms for a ticket (BS_ERR_TIMEOUT after that). */
int bs_server_wait(bs_server *s, uint64_t ticket, int32_t timeout_ms, bs_query_result *res);

/* Copy the first min(count, cap) values of a completed query to dst (device
 * memory or pinned host memory), ordered on `stream`. Returns the number of
 * values copied in *copied (may be NULL). NOT_READY if the query is not done. */
int bs_server_copy_result(bs_server *s, uint64_t ticket, int32_t *dst, uint64_t cap, uint64_t *copied,
                          void *stream);

/* Free a completed query's result buffer (its d_values become invalid). */
int bs_server_release(bs_server *s, uint64_t ticket);

int bs_server_get_stats(const bs_server *s, bs_server_stats *st);

/* Test hook (the paper has no counterpart): the next n batch launches of this
 * server fail on the host with BS_ERR_CUDA before anything is enqueued, as a
 * refused launch would; their queries complete with that status. */
int bs_server_fail_next_launches(bs_server *s, int32_t n);

/* Stops the dispatcher after the batches in flight finish, frees everything. */
void bs_server_destroy(bs_server *s);

/* -------------------------------------------------------- diagnostics */

const char *bs_strerror(int status);

/* Test hook (the paper has no counterpart): one device thread waits for a flag
 * that nothing sets, with the same bounded wait the batched kernel's grid
 * barrier uses (at most max_polls polls, max_polls <= 2^24). *gave_up = 1 when
 * the wait gave up as it must; it also leaves a timeout in the device status
 * word, which the next bs_last_device_error reports as BS_ERR_TIMEOUT. Errors:
 * INVALID_ARG, OOM, CUDA. */
int bs_selftest_bounded_wait(uint32_t max_polls, int32_t *gave_up);

/* Reads and clears the device status word of the current device (a kernel
 * bounds check or a bounded wait that gave up). Synchronises the device.
 * Returns BS_OK, BS_ERR_DEVICE_CHECK or BS_ERR_TIMEOUT. */
int bs_last_device_error(void);

/* Library version string. */
const char *bs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BYTESTORE_H */

/*
 * rmq.h -- C ABI of the GB300 batched range-minimum-query library
 * (librmq_gb300.so, CUDA for sm_103a).
 *
 * Method: the block-based sparse table (BbST) of S. Grabowski and
 * T. Kowalski, "Faster batched range minimum queries" (arXiv:1706.06940),
 * in its two forms:
 *   - plain BbST (Sec. 3.2): blocks of k cells over A, a sparse table over
 *     the block minima (Sec. 3.1 step 3), and query answering with two table
 *     lookups plus speculative reads of the two end blocks (Sec. 3.1 step 4);
 *   - contracted BbST_CON (Sec. 3.1): sort the 2q query endpoints (step 1),
 *     contract A to the minima between consecutive endpoints (step 2), then
 *     steps 3 and 4 over the contracted array A_Q.
 *
 * Problem (Sec. 1): for an int32 array A[0..n) and queries [l_i, r_i],
 * out_i = the position of the minimum of A[l_i .. r_i].  This library uses
 * 0-based inclusive ranges and always returns the LEFTMOST minimum position,
 * so every valid answer is unique and bit-exact, independent of k, of the
 * form used and of batching.
 *
 * Conventions for every entry point:
 *   - Pointers named A, l, r, out, T, P, ... are DEVICE pointers owned by the
 *     caller unless a name ends in _host.  Nothing is retained after return
 *     except where a handle says so (rmq_build borrows A).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Device work is enqueued on it and the call returns without
 *     waiting, except rmq_batch_host and rmq_stream_status, which wait.
 *   - Host-detectable errors (null pointer with a non-zero size, n <= 0,
 *     n or q too large, a bad block size) return immediately and enqueue
 *     nothing.  A failed CUDA call returns RMQ_ERR_CUDA; workspace exhaustion
 *     returns RMQ_ERR_OOM.
 *   - A query with l < 0, r >= n or l > r is invalid: its out entry is set
 *     to -1 on the device and a sticky device error word is raised, which
 *     rmq_stream_status reports as RMQ_ERR_QUERY_RANGE.  l and r are never
 *     swapped.
 *   - Sizes: 1 <= n <= 2^31 - 1, 0 <= q <= 2^31 - 1 (q == 0 is a no-op).
 *   - A is int32; arrays that are 16-byte aligned are read with 128-bit
 *     loads, others with 32-bit loads (same results).
 *   - Workspace comes from the device's stream-ordered memory pool
 *     (cudaMallocAsync on `stream`), so calls can be captured in a CUDA graph.
 *   - Calls are thread-safe on distinct handles and buffers.
 *
 * Packed keys: tables produced by the step-level entry points hold uint64
 *   key(i) = ((uint64)((uint32)A[i] ^ 0x80000000) << 32) | (uint32)i
 * whose unsigned order is (value, position) order, so the minimum key is the
 * leftmost minimum and its low 32 bits are the position.
 */
#ifndef RMQ_GB300_H
#define RMQ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmq_handle_s *rmq_handle;   /* opaque, owned by the library */

typedef enum {
    RMQ_OK = 0,
    RMQ_ERR_INVALID_ARG = 1,   /* bad pointer, size or option; nothing enqueued */
    RMQ_ERR_QUERY_RANGE = 2,   /* at least one query had l < 0, r >= n or l > r */
    RMQ_ERR_OOM = 3,           /* device memory for workspace or a handle ran out */
    RMQ_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    RMQ_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    RMQ_ERR_BUDGET = 6,        /* a memory budget set by the caller would be exceeded */
    RMQ_ERR_SCRATCH_LIMIT = 7  /* rmq_batch_noalloc: the table does not fit its fixed buffer */
} rmq_status;

typedef enum {
    RMQ_VARIANT_AUTO = 0,        /* the tuner picks (rmq_tune) */
    RMQ_VARIANT_PLAIN = 1,       /* BbST without contraction (Sec. 3.2) */
    RMQ_VARIANT_CONTRACTED = 2   /* BbST_CON (Sec. 3.1) */
} rmq_variant;

/* rmq_opts.flags bits. */
#define RMQ_FLAG_TEST_WITHHOLD_READY 1u  /* rmq_batch_multi test hook: array 0's table is never
                                            marked ready, so its queries time out (answers -1,
                                            RMQ_ERR_TIMEOUT) after a short bounded wait */

/* Options; a NULL rmq_opts* means all defaults (zeros). */
typedef struct {
    int32_t variant;   /* rmq_variant */
    int32_t k;         /* block size over A (plain form): 0 = tuned, else a power of 2 in [32, 65536] */
    int32_t k_con;     /* block size over A_Q (contracted form): 0 = tuned, else a power of 2 in [32, 65536] */
    int32_t flags;     /* 0, or RMQ_FLAG_* bits where an entry point allows them */
    int32_t threads_per_query;  /* lanes that scan one partial block of an open query (Sec. 3.1 step 4):
                                   0 = tuned (default: teams of 8, 16 or 32 lanes by scan length),
                                   8, 16 or 32 = teams of at least that many lanes */
    int32_t k1;        /* small blocks of the two-level layout (Sec. 3.3), plain form: 0 = tuned
                          (default: 128 cells when k >= 128, none below), -1 = none, else a power
                          of 2 in [32, k]: the minima of every k1 cells are kept beside the block
                          table, and a partial block is resolved from them plus at most two
                          parts of k1 cells */
} rmq_opts;

/* One array of a multi-array batch: A is a device pointer to n int32 cells;
 * the array's q queries are the next q entries of the batch's l, r, out. */
typedef struct {
    const int32_t *A;
    int64_t n;
    int64_t q;
} rmq_array;

/* Capacity of the fixed table buffer of rmq_batch_noalloc, in 8-byte entries
 * (4 MiB; the buffer also holds the table's 32 KiB coarse summary). */
#define RMQ_NOALLOC_TABLE_ENTRIES (1 << 19)

/* ------------------------------------------------------------------ batch */

/* Answer q queries over A in one pass (Sec. 3.1 / 3.2): out[i] = leftmost
 * argmin of A[l[i] .. r[i]].  Form and block size are tuned for (n, q).
 * A: int32[n]; l, r, out: int32[q]. */
rmq_status rmq_batch(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                     int64_t q, int32_t *out, void *stream);

/* rmq_batch with explicit options (form, k, k_con). */
rmq_status rmq_batch_ex(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                        int64_t q, int32_t *out, const rmq_opts *opts, void *stream);

/* rmq_batch_ex that also records CUDA events on `stream` at the stage
 * boundaries of the method, for per-stage timing (the breakdown of Table 1).
 * events: cudaEvent_t handles created by the caller (passed as void*).
 * Plain form (Sec. 3.2), 4 events: start | block minima | sparse table |
 *   queries.
 * Contracted form (Sec. 3.1), 6 events: start | step 1 sort | step 1 remap |
 *   step 2 contraction | step 3 block minima and table over A_Q | step 4;
 *   a 7th event, if given, is recorded inside step 1's sort, after the
 *   clearing of the endpoint bitmap and before the marking of the endpoints.
 * With fewer events only the first n_events boundaries are recorded. */
rmq_status rmq_batch_timed(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                           int64_t q, int32_t *out, const rmq_opts *opts, void *stream,
                           void *const *events, int32_t n_events);

/* rmq_batch_ex on HOST buffers: copies A, l, r to the device, answers, copies
 * out back, and returns after out_host is written (synchronous).  Host
 * buffers may be pageable or pinned; pinned ones copy faster.  Device
 * buffers come from the stream-ordered pool.  Invalid queries answer -1; the
 * call returns what rmq_stream_status returns after the batch (the device
 * error word, so RMQ_ERR_QUERY_RANGE for invalid queries), and clears it. */
rmq_status rmq_batch_host(const int32_t *A_host, int64_t n, const int32_t *l_host,
                          const int32_t *r_host, int64_t q, int32_t *out_host,
                          const rmq_opts *opts, void *stream);

/* Work that the queries left open by the coarse level did, as counted by
 * rmq_batch_counted.  scan_elems is the S of the algorithmic-bytes model:
 * elements read by partial-block scans (Sec. 3.1 step 4), int32 cells of A
 * for the plain form, 8-byte keys of A_Q for the contracted form. */
typedef struct {
    int64_t open_queries;  /* queries finished on the block table (not settled by the coarse level) */
    int64_t table_reads;   /* 8-byte block-table entries they gathered */
    int64_t m1_reads;      /* 8-byte small-block minima they read (plain form, k >= 128; Sec. 3.3) */
    int64_t scan_elems;    /* elements read by partial-block scans (whole 16-byte vectors) */
    int64_t rank_reads;    /* 4-byte endpoint-bitmap words and counts read for their ranks (contracted) */
} rmq_scan_stats;

/* rmq_batch_ex through an instrumented query kernel that also counts the
 * work of its open queries into *stats (host), for the measurement of the
 * edge-scan bytes; answers are the same as rmq_batch_ex's.  Slower than
 * rmq_batch_ex (a measurement tool, not a serving path); waits for the
 * stream.  A, l, r and out must be 16-byte aligned (RMQ_ERR_INVALID_ARG
 * otherwise). */
rmq_status rmq_batch_counted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                             int64_t q, int32_t *out, const rmq_opts *opts, void *stream,
                             rmq_scan_stats *stats);

/* Plain-BbST batch that allocates no device memory (the paper has no
 * counterpart: this is a deployment variant of rmq_batch_ex with the plain
 * form).  Some callers cannot call cudaMalloc: hosts that reserve all device
 * memory for their own allocator up front, and loops that forbid allocation
 * after start-up because it can synchronise the device and take unbounded
 * time.  This entry point keeps the sparse table in a fixed buffer of
 * RMQ_NOALLOC_TABLE_ENTRIES entries (4 MiB, plus 32 KiB for the table's
 * coarse summary) inside the library's device image,
 * held on every GPU that loads the library until the process exits; it calls
 * no cudaMalloc, cudaFree or other allocating routine.  The caller passes A, l,
 * r and out as for rmq_batch_ex.
 *   k: block size, a power of 2 in [32, 65536], or 0 for the tuned k, raised
 *      (doubled) until the table fits.
 *   Returns RMQ_ERR_SCRATCH_LIMIT, enqueuing nothing, when the table for (n, k)
 *   needs more than RMQ_NOALLOC_TABLE_ENTRIES entries (rmq_table_bytes(n, k) / 8).
 * The first call on a device looks up the buffer's device address (once per
 * device, with that device current).  That lookup loads the library's module
 * on the device, which is when the driver commits the buffer's memory: make
 * the first call at start-up, before the caller's allocator takes the rest of
 * device memory and before any stream capture.  A call with q == 0 (l, r, out
 * may be NULL) performs only this set-up.  All calls on a device share the one buffer, and every entry a call
 * reads is written by that call first, so leftovers of earlier calls do not
 * matter; but calls whose work overlaps on the GPU (other streams, or other
 * threads) race on the buffer and must be serialised by the caller. */
rmq_status rmq_batch_noalloc(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                             int64_t q, int32_t *out, int32_t k, void *stream);

/* Many independent arrays, each with its own queries, answered in ONE
 * persistent kernel launch (plain BbST per array, Sec. 3.2, with a coarse
 * level as in Sec. 3.3): block minima, tables and answers for every array.
 * arrays: host array of H descriptors (A device pointers, n >= 1 when q > 0,
 * q >= 0).  The queries of array h are l/r/out entries [s_h, s_h + q_h) with
 * s_h = q_0 + ... + q_{h-1}; their positions are relative to array h, and so
 * are the answers.  Invalid queries answer -1 (RMQ_ERR_QUERY_RANGE via
 * rmq_stream_status).  opts->k forces one block size for every array (0 =
 * chosen per array; at most 32768 here); opts->variant is ignored; opts->flags may hold
 * RMQ_FLAG_TEST_WITHHOLD_READY.  Workspace comes from the stream-ordered pool
 * and the call only enqueues memsets and kernel launches, so it can be
 * captured in a CUDA graph.  Arrays beyond 1024 are handled by further
 * launches of the same kernel. */
rmq_status rmq_batch_multi(const rmq_array *arrays, int32_t H, const int32_t *l, const int32_t *r,
                           int32_t *out, const rmq_opts *opts, void *stream);

/* -------------------------------------------------------- resident arrays */

/* Build the plain-BbST state of A (Sec. 3.2: block minima and their sparse
 * table) and keep it resident in a handle.  A is BORROWED: it must stay
 * alive and unmodified until rmq_free.  The build is enqueued on `stream`;
 * queries on another stream must be ordered after it by the caller.
 * opts->variant is ignored (handles are always plain); opts->k picks k. */
rmq_status rmq_build(const int32_t *A, int64_t n, const rmq_opts *opts, void *stream,
                     rmq_handle *out_handle);

/* Answer q queries against a built handle (Sec. 3.1 step 4 only). */
rmq_status rmq_query(rmq_handle h, const int32_t *l, const int32_t *r, int64_t q,
                     int32_t *out, void *stream);

/* rmq_query on HOST buffers (pageable or pinned): copies l, r to the device,
 * answers, copies out back and returns after out_host is written
 * (synchronous); one request per call.  Device buffers come from the
 * stream-ordered pool.  Returns what rmq_stream_status returns after the
 * call (RMQ_ERR_QUERY_RANGE for invalid queries, which answer -1). */
rmq_status rmq_query_host(rmq_handle h, const int32_t *l_host, const int32_t *r_host, int64_t q,
                          int32_t *out_host, void *stream);

/* Queries of H requests against resident handles in ONE kernel launch:
 * request h asks q_counts[h] queries (consecutive in l, r, out; positions
 * relative to hs[h]'s array).  A handle may appear in several requests.
 * q_counts: host array.  Invalid queries answer -1.  Graph-capturable. */
rmq_status rmq_query_multi(const rmq_handle *hs, const int64_t *q_counts, int32_t H, const int32_t *l,
                           const int32_t *r, int32_t *out, void *stream);

/* Device bytes owned by the handle (its sparse table), 0 for NULL. */
int64_t rmq_handle_bytes(rmq_handle h);

/* Block size k of the handle, 0 for NULL. */
int32_t rmq_handle_k(rmq_handle h);

/* Release a handle (waits for the device work that uses it). NULL is a no-op. */
void rmq_free(rmq_handle h);

/* ---------------------------------------------------------------- serving
 * A continuous-batching request server over resident arrays (host threads
 * inside the library).  An array holds 4n bytes plus exactly the tables
 * rmq_build allocates for it (rmq_handle_bytes) against the memory budget.
 * Each submitted request (an array id and HOST buffers l, r, out of q
 * entries) is queued; a scheduler thread packs all pending requests into one
 * batch per tick and runs it on one of several streams (upload, one
 * multi-request query launch, download) while earlier batches are still
 * running; a completion thread copies the answers into the requests' out
 * buffers.  The caller keeps l, r, out alive and unmodified until
 * rmq_server_wait returns for the ticket.  A request's array stays resident
 * from submit until its answers are copied: rmq_server_evict waits for that. */
typedef struct rmq_server_s *rmq_server;

typedef struct {
    int64_t budget_bytes;       /* device bytes for resident arrays and tables; 0 = no limit */
    int32_t inflight;           /* batches on the GPU at once (streams); 0 = 4 */
    int32_t max_batch_queries;  /* queries per batch and per request at most; 0 = 4194304 */
    int32_t flags;              /* reserved, must be 0 */
    int32_t pad;
} rmq_server_opts;

typedef struct {
    int64_t requests;            /* completed requests */
    int64_t queries;             /* their queries */
    int64_t batches;             /* batches launched */
    int64_t table_bytes_in_use;  /* bytes reserved for resident arrays and tables */
    int64_t resident_arrays;
} rmq_server_stats;

/* Create a server on the current device. */
rmq_status rmq_server_create(const rmq_server_opts *opts, rmq_server *out);

/* Build and keep resident the plain-BbST state of device array A (borrowed,
 * like rmq_build); k = 0 picks it.  The build runs on the server's own stream,
 * so A must be completely written before the call (synchronize the stream
 * that wrote it).  Waits for the build.  RMQ_ERR_BUDGET (and nothing is
 * built) when it does not fit the budget now; RMQ_ERR_OOM when the device
 * has no memory left for its tables. */
rmq_status rmq_server_admit(rmq_server s, const int32_t *A, int64_t n, int32_t k, int32_t *id_out);

/* rmq_server_admit that, when the array does not fit the budget now, waits
 * up to timeout_s seconds for evictions to free enough of it (RMQ_ERR_BUDGET
 * if they do not, or at once if the array alone exceeds the budget). */
rmq_status rmq_server_admit_wait(rmq_server s, const int32_t *A, int64_t n, int32_t k, double timeout_s,
                                 int32_t *id_out);

/* Release an array's tables.  From the call on, new requests on id are
 * refused (RMQ_ERR_INVALID_ARG); the call waits until every request already
 * submitted on id has completed, then frees the tables.  RMQ_ERR_INVALID_ARG
 * for an unknown id or one already being evicted. */
rmq_status rmq_server_evict(rmq_server s, int32_t id);

/* Queue a request of q queries on array id; returns a ticket at once.
 * RMQ_ERR_INVALID_ARG for an unknown or evicted id, or q above the server's
 * max_batch_queries. */
rmq_status rmq_server_submit(rmq_server s, int32_t id, const int32_t *l_host, const int32_t *r_host, int64_t q,
                             int32_t *out_host, int64_t *ticket_out);

/* Wait until the ticket's answers are in its out buffer; *latency_s = time
 * from submit to answers (seconds, may be NULL).  Each ticket is waited once:
 * a wait on a ticket that was never issued or has already been collected
 * returns RMQ_ERR_INVALID_ARG at once.  Returns RMQ_ERR_QUERY_RANGE when some
 * query of this request had l < 0, r >= n or l > r (checked on the host when
 * the request is batched; those answers are -1, the others are valid), and
 * RMQ_ERR_CUDA when its batch failed on the device. */
rmq_status rmq_server_wait(rmq_server s, int64_t ticket, double *latency_s);

rmq_status rmq_server_stats_get(rmq_server s, rmq_server_stats *out);

/* Stop the threads, finish running batches and free everything; requests
 * still queued are not run.  No other thread may be inside an rmq_server_*
 * call on s (a wait included) while it is destroyed, nor call one after. */
void rmq_server_destroy(rmq_server s);

/* ----------------------------------------------------------- diagnostics */

/* Wait for `stream`, then report and clear its sticky device error word:
 * the errors raised by this library's calls on this stream (on the current
 * device) since the last report: RMQ_OK, RMQ_ERR_QUERY_RANGE or
 * RMQ_ERR_TIMEOUT (RMQ_ERR_CUDA if the stream itself failed).  Each stream
 * has a word of its own, so calls on other streams neither raise nor
 * consume it.  NULL and cudaStreamLegacy share the legacy stream's word; a
 * device keeps words for 255 other streams, and streams beyond those share
 * words round-robin. */
rmq_status rmq_stream_status(void *stream);

/* Number of kernel launches this library has issued in the process so far
 * (all devices, all threads); host only. */
int64_t rmq_launch_count(void);

/* Static description of a status code (never NULL). */
const char *rmq_strerror(rmq_status s);

/* Bytes of a plain-BbST sparse table for (n, k): nb * (floor(log2 nb) + 1) * 8
 * with nb = ceil(n / k) (the memory model of Table 2).  -1 on bad arguments. */
int64_t rmq_table_bytes(int64_t n, int32_t k);

/* The plain form over the l-ary block sparse table (the variant of Sec. 3.1
 * that the paper describes without implementing): level t holds the minimum
 * of every l^t consecutive blocks, so a query's inner span is covered by at
 * most l table values, and the table has floor(log_l nb) + 1 levels
 * (nb = ceil(n / k)) instead of floor(log2 nb) + 1.  k: power of two in
 * [32, 65536]; ell: power of two in [2, 256].  Same answers, error behaviour
 * and ownership as rmq_batch_ex; its table (levels * nb * 8 bytes) comes from
 * the stream-ordered pool.  One launch per level, one thread per query. */
rmq_status rmq_batch_lary(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                          int64_t q, int32_t *out, int32_t k, int32_t ell, void *stream);

/* Device workspace, in bytes, that one rmq_batch_ex call with these
 * arguments takes from the stream-ordered pool: the extra memory beside the
 * 4n bytes of A, as Table 2 reports it.  Plain form: levels 0..lc of the
 * block table and, for k >= 128, the minima of every 128 cells.  Contracted
 * form: the endpoint bitmap with rank counts, A_Q (up to min(2q, n) - 1
 * keys), the table over A_Q and the coarse index.  Host only; -1 on bad
 * arguments (those rmq_batch_ex rejects). */
int64_t rmq_batch_workspace_bytes(int64_t n, int64_t q, const rmq_opts *opts);

/* The plain form over the multi-level block-based sparse table of Sec. 3.3.
 * ks[0 .. h-1] = k_1 < k_2 < ... < k_h, host array of powers of two (so each
 * divides the next), 32 <= k_1 <= 65536, k_h <= 2^30, 1 <= h <= 8.  The
 * minima of the blocks of k_i are kept for i < h and a sparse table over the
 * blocks of k_h; a query reads two table values for the whole blocks of k_h
 * inside it and walks each end part down the levels (at most k_h / k_{h-1} +
 * ... + k_2 / k_1 + k_1 reads per end).  h == 1 is the one-level table of
 * Sec. 3.2 with k = k_1.  Same answers, error behaviour and ownership as
 * rmq_batch_ex; the structure (rmq_hlevel_bytes) comes from the
 * stream-ordered pool and is freed when the call's work is done.
 * RMQ_ERR_INVALID_ARG for bad block sizes. */
rmq_status rmq_batch_hlevel(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r,
                            int64_t q, int32_t *out, const int32_t *ks, int32_t h, void *stream);

/* Bytes of the structure rmq_batch_hlevel builds: 8 * (ceil(n/k_1) + ... +
 * ceil(n/k_{h-1}) + nb (floor(log2 nb) + 1)) with nb = ceil(n / k_h), the
 * space of Sec. 3.3.  Host only; -1 on bad arguments. */
int64_t rmq_hlevel_bytes(int64_t n, const int32_t *ks, int32_t h);

/* Sec. 3.3's choice of block sizes for n and h (2 <= h <= 8): k_i =
 * sqrt(n) * log2(n)^((i-1)/(h-1) - 1/(h+1)), each rounded to the nearest
 * power of two, k_1 kept in [32, 65536] and every k_i made at least twice
 * k_{i-1}.  Writes h values to ks_out (host).  Host only. */
rmq_status rmq_hlevel_paper_ks(int64_t n, int32_t h, int32_t *ks_out);

/* The tuner's choice of options for (n, q); host only.  When rmq_autotune
 * has remembered choices for several width classes of this shape, this
 * returns the one of the lowest width class (rmq_tune_batch chooses by a
 * batch's widths).  Without a remembered choice: the plain form with k near
 * sqrt(n)/8 (and k_con near sqrt(2q), at most 512), threads_per_query and k1
 * at their defaults (0). */
rmq_status rmq_tune(int64_t n, int64_t q, rmq_opts *out);

/* The options an AUTO call (rmq_batch, or rmq_batch_ex with zero fields)
 * uses for this batch: the remembered choice for its shape and, when the
 * shape holds choices for several width classes, for the width class of the
 * batch, which is found from 256 of its queries read back to the host (the
 * call then waits for `stream`; calls during stream capture skip the read
 * and take the lowest class).  l, r: device int32[q]. */
rmq_status rmq_tune_batch(const int32_t *l, const int32_t *r, int64_t q, int64_t n, void *stream, rmq_opts *out);

/* Autotuner (the paper leaves automated selection of k open, Sec. 5):
 * times rmq_batch_ex on this batch for every power-of-two block size in
 * [k_min, k_max] (0, 0 = [32, 4096]) and for the form(s) allowed by
 * `variant` (AUTO = both); then, for the fastest, the lanes per partial-block
 * scan (threads_per_query 16 and 32 against the default) and, for the plain
 * form, the small blocks of the two-level layout (k1 none, 32 .. 512, at most
 * k/2, against the default).  Returns the fastest options in *best (and its
 * time in ms in *best_ms, may be NULL).  Each candidate runs once untimed,
 * then three times, each after a read of twice the L2 size has evicted the
 * batch from L2; its time is the best of the three.  `out` receives answers
 * while it measures.  Waits for the device.  With variant == AUTO the choice
 * is remembered for the batch's shape: (round(log2 n), round(log2 q), width
 * class = round(log2 of the median width r - l + 1 of 256 sampled queries)),
 * so that batches of the same n and q but different widths keep separate
 * choices; rmq_tune, rmq_tune_batch, rmq_batch and rmq_build use them from
 * then on. */
rmq_status rmq_autotune(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                        int32_t *out, int32_t variant, int32_t k_min, int32_t k_max, void *stream,
                        rmq_opts *best, float *best_ms);

/* Write / read the remembered choices (text, one per line:
 * "log2n log2q wclass variant k k_con threads_per_query k1"; lines of the
 * older form "log2n log2q variant k k_con" load as choices that serve every
 * width class of their shape).  Loading merges into the current choices. */
rmq_status rmq_tune_save(const char *path);
rmq_status rmq_tune_load(const char *path);

/* Forget every remembered choice. */
void rmq_tune_clear(void);

/* ------------------------------------------- step-level entry points
 * One step of the method each, on caller buffers, for composition and for
 * checking each step on its own.                                          */

/* Sec. 3.1 step 3, level 0: T0[j] = min key over A[j*k .. min(n,(j+1)*k) - 1],
 * j < ceil(n/k).  T0: uint64[ceil(n/k)]. */
rmq_status rmq_block_minima(const int32_t *A, int64_t n, int32_t k, uint64_t *T0,
                            void *stream);

/* Sec. 3.1 step 3, all levels: given level 0 in T[0 .. nb), fill levels
 * t = 1 .. floor(log2 nb): T[t*nb + j] = min(T[(t-1)*nb + j],
 * T[(t-1)*nb + j + 2^(t-1)]) for j + 2^t <= nb (other slots are left as they
 * are).  T: uint64[nb * (floor(log2 nb) + 1)], level-major. */
rmq_status rmq_sparse_table_build(uint64_t *T, int64_t nb, void *stream);

/* Sec. 3.1 step 1: sort the 2q endpoints (position, tag = 2i + side) by
 * position, stably (equal positions keep the order l_0, r_0, l_1, ...).
 * An invalid query (l < 0, r >= n or l > r) takes part as (0, 0) and raises
 * the device error word.  pos_out, tag_out: uint32[2q]. */
rmq_status rmq_sort_endpoints(const int32_t *l, const int32_t *r, int64_t q, int64_t n,
                              uint32_t *pos_out, uint32_t *tag_out, void *stream);

/* Sec. 3.1 step 1 (remapping): from sorted endpoints, P[0 .. m) = distinct
 * positions in increasing order, rank_l[i] / rank_r[i] = index in P of
 * l_i / r_i, and *m_dev = m (a device int64).  P_out: uint32[2q]. */
rmq_status rmq_rank_endpoints(const uint32_t *pos_sorted, const uint32_t *tag_sorted,
                              int64_t q, uint32_t *P_out, int64_t *m_dev,
                              int32_t *rank_l, int32_t *rank_r, void *stream);

/* Sec. 3.1 step 1 as the batch path computes it: a bitmap over the
 * positions of A in place of the sort.  With W = ceil(n/32) + 1, BP is
 * uint32[2W]: BP[w] (w < W) = bit word w (bit b set: position 32w + b is an
 * endpoint of some query; word W-1 is 0), BP[W + w] = number of set bits in
 * words 0 .. w-1 (so BP[2W - 1] = m).  The set bits in increasing order are P
 * of rmq_rank_endpoints, and the rank of an endpoint p is BP[W + p/32] +
 * popcount of the bits of word p/32 below p % 32.  *m_dev (device int64) = m.
 * An invalid query marks position 0 (as the sort's pair (0, 0)) and raises
 * the device error word.  BP must be 4-byte aligned; the call writes all of
 * it. */
rmq_status rmq_endpoint_bitmap(const int32_t *l, const int32_t *r, int64_t q, int64_t n,
                               uint32_t *BP, int64_t *m_dev, void *stream);

/* Sec. 3.1 step 2: A_Q[j] = min key over A[P_j .. P_{j+1}] (both ends
 * included), j < m - 1, where m = *m_dev (device) and m <= m_max (host bound,
 * used to size the launch).  P must be strictly increasing positions < n.
 * AQ: uint64[max(m_max - 1, 1)]. */
rmq_status rmq_contract(const int32_t *A, int64_t n, const uint32_t *P, const int64_t *m_dev,
                        int64_t m_max, uint64_t *AQ, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RMQ_GB300_H */

/*
 * pospopcnt.h -- C ABI of libpospopcnt.so, the GB300 (sm_103a) positional
 * population count.
 *
 * The operation (arXiv 2412.16370, Fig. 2 and Section 1): for an array of
 * n words of w bits, count for every bit position j < w how many words have
 * bit j set.  Equivalently the input bit stream is read as w interleaved
 * streams and the bits at stream positions j, j+w, j+2w, ... are summed.
 *
 * Conventions shared by every entry point below:
 *
 *   - Byte order.  Words are little-endian, so bit j of a word lives in byte
 *     j/8 of that word; for the byte-length forms bit b of byte k is stream
 *     bit 8k+b and is counted in counter (8k+b) mod w.  A trailing partial
 *     word counts as if zero-padded.  The start address may have any byte
 *     alignment.
 *   - Add-into.  Counts are ADDED to the uint64_t counters the caller passes
 *     (Section 4, step 1 and its footnote: clearing the counters is
 *     optional, which lets streamed or non-contiguous input be counted into
 *     one counter array).  Zero them first for a fresh count.
 *   - Widths.  w is 8, 16, 32 or 64 (the paper's f_8 .. f_64, Section 5).
 *     The byte-length, batch, gather and serving forms also accept w = 1, 2,
 *     4 (w = 1 is the ordinary population count); pospopcnt_async,
 *     pospopcnt_host and the batch and gather forms also the wider folds
 *     w = 128 and 256 (Section 4's general maximum word size; counters then
 *     hold 128 or 256 entries per array).
 *   - Memory.  Unless a function says otherwise, pointers are DEVICE
 *     pointers of the current CUDA device (cudaMalloc, PyTorch tensors,
 *     cudaMallocManaged or pinned host memory that the device can address).
 *     A plain pageable host pointer returns POSPOP_EPTR.  The caller owns
 *     inputs and counters; the library owns its workspace.
 *   - Streams.  `stream` is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  *_async and batch calls only enqueue work:
 *     they neither allocate nor synchronise once the workspace is large
 *     enough, so they may be captured into a CUDA graph (see
 *     pospopcnt_reserve).
 *   - Errors.  Functions return POSPOP_OK (0) or a negative POSPOP_E* code;
 *     n == 0 (or m == 0) is a no-op that returns POSPOP_OK.  A failed call
 *     leaves the counters untouched unless it says otherwise.
 */
#ifndef POSPOPCNT_H
#define POSPOPCNT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define POSPOP_OK 0
#define POSPOP_EINVAL (-1)    /* bad argument: NULL with n > 0, bad w, decreasing offsets */
#define POSPOP_EPTR (-2)      /* pointer not addressable by the device (or wrong kind) */
#define POSPOP_ECUDA (-3)     /* a CUDA runtime call or a kernel launch failed */
#define POSPOP_ENOMEM (-4)    /* workspace or staging memory could not be allocated */
#define POSPOP_ETIMEDOUT (-5) /* a bounded wait expired */
#define POSPOP_EBUSY (-6)     /* no free slot / budget (serving) */
#define POSPOP_ERANGE (-7)    /* size beyond a documented maximum */

/* Message for a status code (static storage, never NULL). */
const char *pospopcnt_strerror(int code);

/* Set up the library for `device` (workspace, launch table, tune table) and
 * make it the current device of the calling thread.  Idempotent.  Other
 * entry points set up the current device on first use, so calling this is
 * optional; call it before capturing a CUDA graph. */
int pospopcnt_init(int device);

/* Release every device's workspace and staging buffers.  Later calls set
 * the library up again. */
void pospopcnt_shutdown(void);

/*
 * Fig. 2's pospop_w(counts, words, n) for w = 8, 16, 32, 64: counts[j] +=
 * number of the n words with bit j set.  `counts` and `words` are either
 * both device-addressable pointers (the count runs on the legacy default
 * stream) or both plain host pointers (the input is streamed to the device
 * through the library's staging buffers, as pospopcnt_host).  Mixed kinds
 * return POSPOP_EPTR.  These calls return when the counts are final, and
 * report kernel errors.
 */
int pospopcnt_u8(uint64_t counts[8], const uint8_t *words, size_t n);
int pospopcnt_u16(uint64_t counts[16], const uint16_t *words, size_t n);
int pospopcnt_u32(uint64_t counts[32], const uint32_t *words, size_t n);
int pospopcnt_u64(uint64_t counts[64], const uint64_t *words, size_t n);

/*
 * Byte-length form, asynchronous (Fig. 2 / Section 1): counts[0..w-1] +=
 * the width-w positional population count of the nbytes bytes at `bytes`
 * (any alignment; a trailing partial word is zero-padded).  Enqueued on
 * `stream`; the counts are final once the stream reaches this point.
 * Device pointers only.
 */
int pospopcnt_async(int w, uint64_t *counts, const void *bytes, size_t nbytes, void *stream);

/*
 * Batched form: m arrays stored at base + offsets[a] .. base + offsets[a+1]
 * (offsets: m+1 uint64_t byte offsets, non-decreasing, in DEVICE memory).
 * counts is an m x w row-major uint64_t array: counts[a*w + j] += count of
 * position j in array a.  One planning pass and one persistent counting
 * launch on `stream` (Section 4's algorithm per work item; the batching is
 * this library's own).  Decreasing offsets are detected on the device: no
 * counter is changed and the stream's batch status becomes POSPOP_EINVAL
 * (read it with pospopcnt_batch_status).  Zero-length arrays are allowed.
 */
int pospopcnt_batch(int w, uint64_t *counts, const void *base, const uint64_t *offsets,
                    size_t m, void *stream);

/*
 * Several independent counts in one launch (each Fig. 2 / Section 1's
 * byte-length count): for i < n, counts[i][0..w[i]-1] += the width-w[i]
 * count of the nbytes[i] bytes at ptrs[i] (any alignment; a trailing partial
 * word zero-padded).  w, counts, ptrs and nbytes are HOST arrays of n
 * entries; counts[i] and ptrs[i] are device-addressable pointers (counts may
 * alias: counts into one counter array add up).  Widths 1 .. 64.  The work
 * is planned on the host and passed in the kernel's parameter block (no
 * upload, no planning kernels), up to 256 counts per launch (more are split
 * into several launches), so a group of small counts costs about one launch
 * instead of one each.  Every entry is checked before anything is enqueued;
 * on an error nothing is counted.  Asynchronous on `stream`.
 */
int pospopcnt_multi(size_t n, const int *w, uint64_t *const *counts, const void *const *ptrs,
                    const size_t *nbytes, void *stream);

/*
 * Gathered regions (Section 4, step 1 and its footnote: leaving the
 * counters uncleared lets non-contiguous memory regions be counted into one
 * counter array): counts[0..w-1] += the counts of the n regions
 * [ptrs[r], ptrs[r] + lens[r]), each counted as its own word stream (its
 * start fixes its word phase; a trailing partial word is zero-padded).
 * ptrs and lens are DEVICE arrays of n uint64_t; every region must be
 * device-addressable (it is read by the kernel, not checked on the host).
 * Same planning and persistent counting as pospopcnt_batch, and the same
 * per-stream workspace.
 */
int pospopcnt_gather(int w, uint64_t *counts, const uint64_t *ptrs, const uint64_t *lens,
                     size_t n, void *stream);

/*
 * Word-selected count (Section 1's GROUP BY count with a WHERE filter):
 * counts[j] += number of words i < n with bit i of `select` set and bit j
 * of word i set, w = 8, 16, 32 or 64.  Bit i of the selection bitmap is bit
 * i % 8 of byte i / 8; the bitmap is read in whole 32-bit words, so
 * 4 * ceil(n / 32) bytes must be readable (bits past n are ignored).
 * `words` must be aligned to the word size and `select` to 4 bytes (else
 * POSPOP_EINVAL).  Device pointers, asynchronous on `stream`.
 */
int pospopcnt_masked(int w, uint64_t *counts, const void *words, size_t n, const void *select,
                     void *stream);

/*
 * pospopcnt_batch for callers that cannot allocate device memory: code
 * recording a CUDA graph in a capture mode that rejects allocation, services
 * that must keep a fixed memory footprint once running, programs whose device
 * memory belongs to another allocator.  The paper has no counterpart; this
 * is a property of this library's batching.
 *
 * Same arguments (w from 1 to 64), kernels and results as pospopcnt_batch,
 * but the work plan
 * lives in a fixed array of the library's own device image (about 513 KiB,
 * held by every GPU that loads the library until the process exits) instead
 * of a cudaMalloc'ed workspace: no call allocates or frees anything.  Limit:
 * m <= 65535 arrays, else POSPOP_ERANGE.  The library looks the array's
 * address up when it sets a device up (pospopcnt_init, or the first call of
 * any entry point on that device), with that device current; make that
 * first call before capturing any stream.  Every call shares the array, so calls that overlap on the GPU
 * (two streams at once, unordered host threads) race and give wrong counts:
 * order them.  Decreasing offsets leave the counters untouched (no status is
 * reported; use pospopcnt_batch to get one).
 */
int pospopcnt_batch_noalloc(int w, uint64_t *counts, const void *base, const uint64_t *offsets,
                            size_t m, void *stream);

/* Synchronise `stream` and return (then clear) the device-side status word of
 * `stream`, set by the batched, gathered, selected and roofline calls on it
 * since it was last read: POSPOP_OK, POSPOP_EINVAL (decreasing offsets) or
 * POSPOP_ETIMEDOUT (a staging wait of the bulk-copy roofline kernel or of
 * the staged selected count expired; see the tune entry `wait`). */
int pospopcnt_batch_status(void *stream);

/* Grow the workspace of `stream` so that batch calls with up to m_max
 * arrays need no allocation (required before capturing such calls into a
 * CUDA graph of the caller's; a capture that needs more returns
 * POSPOP_ENOMEM).  A workspace that was used while its stream was being
 * captured is never freed while the library is set up: when a later call
 * needs a larger one, the old buffer is kept (the caller's graph still
 * replays into it) until pospopcnt_shutdown, so destroy such graphs before
 * shutting down.  A caller's graph reports its status through
 * pospopcnt_batch_status of the capture stream only while that stream's
 * workspace has not been replaced. */
int pospopcnt_reserve(size_t m_max, void *stream);

/*
 * Host-memory form: counts (host, w entries) += the count of the nbytes
 * host bytes at `bytes`.  Pinned host memory is read by the counting kernel
 * directly over the CPU-GPU link; pageable memory is copied through the
 * library's double-buffered device staging area, copies overlapping the
 * counting.  Synchronous.
 */
int pospopcnt_host(int w, uint64_t *counts, const void *bytes, size_t nbytes);

/*
 * Roofline read kernel (the paper's "dummy" kernel of Section 5: it sums
 * the input and adds the sum to an output).  *sum (device, one uint64_t) +=
 * the exact sum (mod 2^64) of the 32-bit little-endian words of the
 * 16-byte-aligned interior of [bytes, bytes + nbytes).  The tune table's
 * `roofline` entry picks the form: direct loads exactly like the counting
 * kernel's (load variants 0 and 1), or staging through shared memory with
 * cp.async.bulk (load variant 2; an expired staging wait is reported by
 * pospopcnt_batch_status).  It is the achievable-bandwidth reference for the
 * counting kernels.
 */
int pospopcnt_roofline_read(const void *bytes, size_t nbytes, uint64_t *sum, void *stream);

/*
 * Launch plan of the single-array count for (w, nbytes) on the current
 * device, as chosen from the tune table.  Writes 8 values to plan:
 * [0] grid blocks, [1] threads per block, [2] CSA flush depth (16 or 32
 * words per a16 flush), [3] load variant, [4] size class, [5] rows of 512 B,
 * [6] launches, [7] resident blocks per SM.  For tests and benchmarks.
 */
int pospopcnt_plan(int w, size_t nbytes, uint32_t plan[8]);

/*
 * Tune table.  A device starts with the table in the file named by the
 * environment variable POSPOP_TUNE_FILE, else pospopcnt_tune.txt next to
 * the library, else built-in defaults.  pospopcnt_autotune times every launch
 * candidate (block shape, CSA flush depth, load variant, blocks per SM, rows
 * per warp; for the batched call work-item rows and grab size) for each width
 * group (w <= 8, 16, 32, >= 64) and, for the single-array count, each size
 * class on the current device (allocating a scratch buffer of up to
 * max_bytes), installs the fastest, and, if path is not NULL, writes the
 * table there.  The table's `wait <cycles>` entry (0 .. 2^31, default 2^31,
 * about a second) bounds how long a staged kernel waits for one bulk copy
 * before it reports POSPOP_ETIMEDOUT and leaves; 0 makes every such wait
 * give up at once (a way to exercise that exit on healthy copies).  pospopcnt_tune_load installs a table
 * written earlier; pospopcnt_tune_describe writes the current table, in the
 * same text format, into buf.
 */
int pospopcnt_autotune(size_t max_bytes, const char *path);
int pospopcnt_tune_load(const char *path);
int pospopcnt_tune_describe(char *buf, size_t len);

/*
 * Check a tune file without a GPU: parse `path` as pospopcnt_tune_load
 * would (same format and limits) and install nothing.  Needs no device and
 * makes no CUDA call.  Returns POSPOP_OK, or POSPOP_EINVAL with *bad_line
 * (if not NULL) set to the 1-based number of the first line that does not
 * parse, 0 when the file cannot be read.
 */
int pospopcnt_tune_check(const char *path, int *bad_line);

/*
 * CUDA graph of one batched call (planning + counting), captured on
 * `stream` (not the legacy stream, and not a stream already being captured)
 * and replayed with pospopcnt_graph_launch on any stream of the same
 * device.  The graph keeps the pointers, w and m it was made with, and owns
 * its scratch memory: a workspace for m arrays allocated when the graph is
 * made and freed by pospopcnt_graph_destroy (which first waits for the last
 * replay to finish).  No other call of the library frees or reuses it, not
 * even pospopcnt_shutdown, so a graph stays valid until it is destroyed.
 * Replays of one graph must not overlap on the GPU (they share its
 * scratch).  *graph receives an opaque handle.
 */
int pospopcnt_batch_graph_create(int w, uint64_t *counts, const void *base,
                                 const uint64_t *offsets, size_t m, void *stream,
                                 void **graph);
int pospopcnt_graph_launch(void *graph, void *stream);
/* Wait for the graph's last replay and return (then clear) its device-side
 * status word: POSPOP_OK, or POSPOP_EINVAL if a replay found decreasing
 * offsets (that replay changed no counter). */
int pospopcnt_graph_status(void *graph);
/* The graph's own scratch memory: device address and size in bytes (either
 * pointer may be NULL).  Fixed for the graph's lifetime. */
int pospopcnt_graph_workspace(void *graph, void **addr, size_t *bytes);
int pospopcnt_graph_destroy(void *graph);

/*
 * ---------------------------------------------------------------------------
 * Serving: continuous batching of pospopcnt requests.  The paper has no
 * serving layer; each request is the byte-length count above (Fig. 2 /
 * Section 1) of device-resident input, and the batching is this library's.
 *
 * A request is admitted when the input bytes of all admitted, unfinished
 * requests plus its own fit `mem_budget` and fewer than `max_inflight` are
 * admitted (and, in modes 1 to 3, at most 16384 at once).  The tune
 * table's `serve_mode` entry, read when a server is created, picks one of
 * four schedules.
 *
 * `serve_mode 1` (the default): admitted requests are ordered by the bytes
 * they still have to count, and whenever one of the server's highest-
 * priority streams is free (`serve_srf`'s <launches> of them, at most
 * `max_batches`) a launch takes work items of the smallest first, up to
 * <bytes> of them, so a large request is counted over several launches and
 * smaller arrivals overtake it at the next launch.  Each request keeps one
 * server-wide slot of counters until its last item is done.  Under load a
 * request's work items have its size class's `serve_srf_class` rows, or
 * else `serve_srf`'s <rows> (modes 2 and 3 likewise).  With `serve_srf_age`
 * set, the longest-waiting request, once it has waited that long, takes up
 * to half of the next launch ahead of the order (off by default).
 *
 * `serve_mode 2`: the same, per size class of the bytes a request has left
 * (the classes below): a launch takes requests of one class only and runs
 * on one of that class's <launches> streams, whose priority falls as the
 * class grows, so blocks of smaller work overtake waiting blocks of larger
 * work on the device.
 *
 * `serve_mode 3`: the order of mode 1 without a launch per batch.  One
 * resident grid on every SM takes work items from a queue in device memory,
 * item by item, and the server publishes runs of the smallest-remaining
 * requests' items into that queue (through mapped host memory) whenever
 * its unclaimed work is below `serve_srf`'s <bytes>.  The grid is launched
 * when work arrives and told to leave after `serve_resident`'s idle time
 * without work; it also leaves by itself after the entry's wait time
 * without a new run, and then the requests it had not finished fail with
 * POSPOP_ETIMEDOUT.  While the grid runs it holds every SM, so other
 * kernels on the device start only after the server has been idle that
 * long.
 *
 * `serve_mode 0`: admitted requests fall into size classes (below 1 MiB,
 * 16 MiB, 128 MiB, and above; as many classes as the device has stream
 * priority levels, at most four), and each class has `max_batches` streams
 * with a priority that falls as the class grows.  A class's admitted
 * requests are gathered into one batch as soon as one of its streams is
 * free, so requests arriving while others run are counted in the next batch
 * while earlier batches are still on the device, and blocks of a smaller
 * class run before waiting blocks of a larger one.  The tune table's `serve`
 * entry of each class sets its work-item rows (while the server is lightly
 * loaded, and otherwise), how many of its batches may run at once (at most
 * `max_batches`) and how many requests a batch takes (at most 1024).
 *
 * In every mode `serve_light` sets the in-flight bytes below which the
 * server counts as lightly loaded (work items then spread a request over
 * every SM), each result is the same as the request's single-array count,
 * and waits are bounded by the caller's timeouts.
 * ---------------------------------------------------------------------------
 */
typedef struct pospop_server pospop_server;

typedef struct pospop_completion {
  uint64_t id;           /* from pospop_server_submit */
  int32_t status;        /* POSPOP_OK, or the error that ended the request */
  int32_t w;
  uint64_t nbytes;
  int64_t t_submit_ns;   /* steady-clock timestamps (nanoseconds) */
  int64_t t_admit_ns;
  int64_t t_launch_ns;
  int64_t t_done_ns;
} pospop_completion;

/* Start a server on the current device (its own streams, pinned staging
 * and device counters; a host thread runs the loop).  mem_budget > 0 bytes,
 * 1 <= max_inflight <= 2^20, 1 <= max_batches <= 64. */
int pospop_server_create(size_t mem_budget, int max_inflight, int max_batches,
                         pospop_server **out);

/* A server as pospop_server_create, that also owns a device staging pool of
 * mem_budget bytes, allocated here once and freed by pospop_server_destroy,
 * for requests whose input is in host memory (pospop_server_submit_host).
 * Such a request is admitted only when a contiguous range of the pool (first
 * fit, in 256-byte granules) is free for it, as well as the budget and slot
 * conditions above, so the budget bounds device memory that is really
 * allocated.  Once admitted, the server's uploader thread copies the input
 * into its range (cudaMemcpyAsync on the server's copy stream), the request's
 * batch waits for that copy, and the range is released when the request
 * completes.  POSPOP_ENOMEM if the pool cannot be allocated. */
int pospop_server_create_pooled(size_t mem_budget, int max_inflight, int max_batches,
                                pospop_server **out);

/* Queue one request whose nbytes of input are in HOST memory at `bytes`
 * (pinned or pageable; it must stay valid and unchanged until the request
 * completes): staged into the server's pool, then counted as by
 * pospop_server_submit.  Only for a server made by
 * pospop_server_create_pooled (else POSPOP_EINVAL); nbytes > mem_budget
 * returns POSPOP_ERANGE; a device or managed pointer returns POSPOP_EPTR.
 * Never blocks. */
int pospop_server_submit_host(pospop_server *s, int w, const void *bytes, size_t nbytes,
                              uint64_t *result, uint64_t *id);

/* Staging pool of a pooled server: stats[0] its bytes, stats[1] bytes held
 * by admitted, unfinished host requests now, stats[2] the most ever held at
 * once (never more than stats[0]).  All zero for a server without a pool. */
int pospop_server_pool_stats(pospop_server *s, uint64_t stats[3]);

/* Queue one request: count the nbytes device-addressable bytes at `bytes`
 * with width w (1, 2, 4, 8, 16, 32, 64).  When it completes, result[0..w-1]
 * (host memory, valid until then; may be NULL) is OVERWRITTEN with the
 * counts.  Never blocks.  nbytes > mem_budget returns POSPOP_ERANGE; a plain
 * host pointer returns POSPOP_EPTR.  *id (may be NULL) receives the id. */
int pospop_server_submit(pospop_server *s, int w, const void *bytes, size_t nbytes,
                         uint64_t *result, uint64_t *id);

/* Move up to max finished requests' records to out, waiting up to
 * timeout_ms for the first.  Returns how many (>= 1) or POSPOP_ETIMEDOUT. */
int pospop_server_poll(pospop_server *s, pospop_completion *out, int max, int timeout_ms);

/* Wait up to timeout_ms until every submitted request has finished. */
int pospop_server_drain(pospop_server *s, int timeout_ms);

/* stats: submitted, finished, waiting for admission, admitted and
 * unfinished, their input bytes, last loop error. */
int pospop_server_stats(pospop_server *s, uint64_t stats[6]);

/* Load generator: submit request i at arrival_ns[i] nanoseconds after the
 * call starts (w[i], device address ptrs[i], nbytes[i], counts into
 * results + 64*i), then collect all n completion records into out[i] (the
 * server's finished queue must be empty and this the only submitter).
 * Returns POSPOP_ETIMEDOUT if they do not all finish within timeout_ms. */
int pospop_server_run_trace(pospop_server *s, size_t n, const int64_t *arrival_ns,
                            const int32_t *w, const uint64_t *ptrs, const uint64_t *nbytes,
                            uint64_t *results, pospop_completion *out, int timeout_ms);

/* Finish every submitted request, stop the loop and free the server. */
int pospop_server_destroy(pospop_server *s);

/* Number of library kernel launches enqueued by this process so far. */
uint64_t pospopcnt_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* POSPOPCNT_H */

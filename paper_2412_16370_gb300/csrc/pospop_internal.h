// pospop_internal.h -- declarations shared by the library's translation
// units (kernel tables, launch parameters).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pospop {

// Longest wait of a staged kernel for one bulk copy, in SM clock cycles
// (about a second at 2 GHz): the default limit of the first wait on a
// stage, and the fixed limit of the waits that drain a warp's copies still
// in flight before it leaves.
constexpr long long kBulkWaitCycles = 1ll << 31;

// One array (or a piece of one) in 16-byte granule coordinates; see
// pospop_device.cuh for the layout.
struct SpanH {
  const uint8_t *A;
  uint64_t G;
  uint32_t head;
  uint32_t tail;
};

struct StreamParams {
  SpanH s;
  uint64_t row_begin;           // rows [row_begin, row_end) of the span in this launch
  uint64_t row_end;
  unsigned long long *counts;   // w counters (device)
  int w;
  uint32_t rot;                 // (8 * head) mod w
  uint32_t regroup;             // w = 8 warps with <= 3 rows use the per-lane bit regroup
};

// Size classes of the arrays of a batched count, by rows of 512 bytes: at
// most 4 rows (2 KiB), 64 (32 KiB), 2048 (1 MiB), and above.  The tune table
// gives each class its own work-item rows; the planning and counting kernels
// both take an array's class from its row count.
constexpr int kBatchClasses = 4;
__host__ __device__ constexpr int batch_class(uint64_t rows) {
  return rows <= 4 ? 0 : rows <= 64 ? 1 : rows <= 2048 ? 2 : 3;
}

// Sources of a batched count (the template parameter SRC of the batch kernels).
constexpr int kSrcCsr = 0;      // m arrays at base + offsets[a] .. base + offsets[a+1], one w
constexpr int kSrcGather = 2;   // regions ptrs[a], lens[a], all counted into one counter array

struct BatchParams {
  const uint64_t *gptrs;        // gathered regions: start addresses (device array)
  const uint64_t *glens;        //                   byte lengths (device array)
  const uint8_t *base;
  const uint64_t *offsets;      // m + 1 byte offsets (device)
  uint64_t m;
  unsigned long long *counts;   // m * w counters (device)
  int w;
  const uint64_t *item_start;   // m + 1 exclusive prefix sums of work items (workspace)
  unsigned long long *next;     // dynamic work counter (workspace)
  const int *status;            // planning status (workspace)
  uint32_t item_rows[kBatchClasses];   // rows of 512 B per work item, by array size class
  uint32_t grab;                // work items taken per atomic
  uint32_t regroup;             // w = 8 items of <= 3 rows use the per-lane bit regroup
};

// One serving launch: up to kServeMax requests passed by value in the
// kernel's parameter block (no upload copy), their work-item prefix sums,
// and the per-request-slot state that the kernel leaves clean for reuse:
// counters (read and cleared by the warp that finishes a request) and
// completion counters (reset by the same warp).
constexpr int kServeMax = 256;

struct ServeReq {
  const void *ptr;              // first byte (device addressable, any alignment)
  uint64_t nbytes;
  int32_t w;
  uint32_t items;               // work items of the whole request
  unsigned long long *out;      // add-into form (pospopcnt_multi): this count's w counters
  uint32_t item0;               // the request's first work item in this launch (a request's
                                // items may be spread over several launches)
  uint32_t slot;                // request slot (counters, completion counter, result, flag)
  uint32_t seq;                 // value written to the slot's flag when the request completes
  uint32_t rows;                // rows of 512 B per work item of this request
};

template <int N>
struct ServeParamsT {
  uint32_t n;                   // requests in this launch
  uint64_t total;               // work items in this launch
  unsigned long long *counts;   // 64 per request slot (device, zero between uses)
  unsigned int *done;           // finished work items per request slot (device, zero between uses)
  unsigned long long *host_res; // 64 per request slot (mapped pinned host memory)
  unsigned int *flags;          // one per request slot (mapped pinned host memory)
  uint32_t strided;             // 1: item k of a request of K items counts rows k, k + K, ...
                                // (warps on neighbouring items read neighbouring rows);
                                // 0: item k counts rows k * rows .. + rows - 1 (rows: the
                                // request's item rows)
  ServeReq req[N];
  uint64_t item_start[N + 1];
};
using ServeParams = ServeParamsT<kServeMax>;

// Launches of at most kServeSmall requests go out with a parameter block of
// that many entries (about 1 KiB instead of 14 KiB): the driver copies the
// whole block into every launch, and a small block reaches the device
// sooner.  The same kernel, instantiated for both sizes.
constexpr int kServeSmall = 16;
using ServeParamsSmall = ServeParamsT<kServeSmall>;

inline void shrink_params(const ServeParams &P, ServeParamsSmall &S) {
  S.n = P.n;
  S.total = P.total;
  S.counts = P.counts;
  S.done = P.done;
  S.host_res = P.host_res;
  S.flags = P.flags;
  S.strided = P.strided;
  for (uint32_t k = 0; k < P.n; k++) {
    S.req[k] = P.req[k];
    S.item_start[k] = P.item_start[k];
  }
  S.item_start[P.n] = P.item_start[P.n];
}

// serve_mode 3: one resident grid fed through a device-side queue.  The host
// publishes runs of a request's work items into a ring in mapped pinned
// memory and raises `published`; one doorbell warp of the grid copies new
// runs into a device ring, gives each run its first ticket, indexes the
// tickets by blocks of 64 and releases the ticket count; every other warp
// claims tickets one at a time and counts the ticket's item.
struct ResRun {
  const void *ptr;              // the request's first byte (device addressable)
  uint64_t nbytes;              // the request's length
  unsigned long long key;       // device ring: (first ticket << kResNBits) | items of the
                                // run, written last, in one 8-byte store (0: no run)
  int32_t w;
  uint32_t items;               // work items of the whole request
  uint32_t item0;               // the run's first item within the request
  uint32_t n;                   // items in the run, below 2^kResNBits
  uint32_t slot;                // request slot (counters, completion counter, result, flag)
  uint32_t tag;                 // written to the slot's flag when the request completes
  uint32_t rows;                // rows of 512 B per work item
  unsigned int left;            // device ring: items of the run not yet counted
  uint32_t pad[2];
};
static_assert(sizeof(ResRun) == 64, "a run is one 64-byte record");
constexpr int kResNBits = 23;                       // items per run, below 2^23
constexpr unsigned long long kResTicketLimit = 1ull << 40;   // tickets before a reset

struct ResCtl {                 // mapped pinned host memory, one per server
  unsigned long long published; // host: runs published so far (release store)
  unsigned long long stop;      // host: the launch epoch that is to leave
  unsigned long long head_seen; // device: tickets claimed so far (the doorbell's copy)
  unsigned long long copied_seen;   // device: runs copied so far (the doorbell's copy)
};

struct ResState {               // device memory; lives across launches
  unsigned long long head;      // next ticket to claim
  unsigned long long tickets;   // tickets released (every run copied so far)
  unsigned long long copied;    // runs copied
  unsigned long long beat;      // %globaltimer when the doorbell last copied a run
  unsigned int stop;            // 1: the grid is to leave (set by the doorbell)
  unsigned int exited;          // warps that have left this launch
  int status;                   // POSPOP_ETIMEDOUT when a wait for work ran out
  unsigned int pad;
};

struct ResParams {
  const ResRun *hruns;          // the host ring (device address of the mapped memory)
  ResCtl *ctl;                  // device address of the mapped control block
  ResRun *druns;                // the device ring (same length)
  uint32_t *idx;                // ring position of the run holding ticket 64 b, by b
  ResState *st;
  unsigned long long *counts;   // 64 per request slot (device, zero between uses)
  unsigned int *done;           // finished work items per request slot
  unsigned long long *host_res; // 64 per request slot (mapped pinned host memory)
  unsigned int *flags;          // one per request slot (mapped pinned host memory)
  uint32_t C;                   // ring length (power of two)
  uint32_t B;                   // index length (power of two)
  unsigned long long epoch;     // this launch's number (the host stops it by writing it)
  long long wait_ns;            // the doorbell leaves after this long without a new run
};

struct PlanParams {
  const uint64_t *gptrs;        // gathered regions
  const uint64_t *glens;
  const uint64_t *offsets;
  uint64_t m;
  uint64_t base_addr;           // (uint64_t)base, for granule alignment
  uint64_t *item_start;         // m + 1
  uint64_t *block_sum;          // one per planning block
  unsigned long long *next;
  int *status;
  uint32_t item_rows[kBatchClasses];   // rows per work item, by array size class
  uint32_t nblocks;
};

// Word-selected single-array count (the stream kernel's parameters plus the
// selection bitmap).
struct SelectParams {
  StreamParams sp;
  const uint8_t *bits;          // selection bitmap (4-byte aligned)
  uint64_t nbits;               // words
  uint64_t nbytes;              // readable bitmap bytes
  uint32_t wlog;                // log2 of the word size in bytes
  uint64_t chunk0;              // staged form: chunks [chunk0, nstaged) of 16 rows are staged
  uint64_t nstaged;             //   in shared memory (the others are counted from registers)
  uint32_t sel_bytes;           // staged form: bitmap bytes copied per chunk
  const uint8_t *sel_base;      // staged form: the bitmap rounded down to 16 bytes
  int64_t sel_bit0;             // staged form: bit of sel_base where chunk 0's bits start
  int *status;                  // staged form: set to POSPOP_ETIMEDOUT if a wait expires
  long long wait_cycles;        // staged form: limit of a wait for a stage (SM clock cycles)
};

struct RooflineParams {
  const uint8_t *A;             // 16-byte aligned
  uint64_t G;                   // whole granules
  unsigned long long *sum;
  int *status;                  // bulk-copy form: set to POSPOP_ETIMEDOUT if a wait expires
  long long wait_cycles;        // bulk-copy form: limit of a wait for a stage (SM clock cycles)
};

// Kernel variant descriptor.  `fn` is the __global__ function to launch
// with a single by-value parameter struct.
struct Variant {
  const void *fn;
  int bs;       // threads per block
  int minb;     // __launch_bounds__ min blocks per SM
  int depth;    // 16 or 32 vectors per flush
  int hint;     // load variant
  int smem = 0; // dynamic shared memory bytes per block
};

constexpr int kPlanThreads = 1024;
constexpr int kPlanPerThread = 4;
constexpr int kPlanChunk = kPlanThreads * kPlanPerThread;

int stream_variant_count();
const Variant &stream_variant(int i);
int stream256_variant_count();
const Variant &stream256_variant(int i);
int batch_variant_count();
const Variant &batch_variant(int i);
int batch256_variant_count();
const Variant &batch256_variant(int i);
int roofline_variant_count();
const Variant &roofline_variant(int i);

int serve_variant_count();
const Variant &serve_variant(int i);
// the same serving kernels with the small parameter block (same order)
const Variant &serve_small_variant(int i);
// The serving kernel's add-into form (pospopcnt_multi): same launch shapes,
// each count added into its own counters, no completion tracking.
int multi_variant_count();
const Variant &multi_variant(int i);
const Variant &multi_small_variant(int i);
// pospopcnt_multi for groups of large counts: the single-array kernel's
// grid-stride schedule over the group's rows (same order as the stream
// kernel table).
// serve_mode 3's resident grid, one per serving launch shape (same order as
// the serving kernel table).
int resident_variant_count();
const Variant &resident_variant(int i);
int multi_stream_variant_count();
const Variant &multi_stream_variant(int i);
int gather_variant_count();
const Variant &gather_variant(int i);
int gather256_variant_count();
const Variant &gather256_variant(int i);
int select_staged_variant_count();
const Variant &select_staged_variant(int i);
int select_variant_count();
const Variant &select_variant(int i);
const void *plan_items_gather_fn();

const void *plan_items_fn();
const void *plan_scan_fn();
const void *plan_apply_fn();

}  // namespace pospop

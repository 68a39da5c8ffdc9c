// pospop_runtime.h -- host-side runtime state shared by the library's
// translation units (device contexts, tune table, workspaces, launchers).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "pospop_internal.h"

namespace pospop {

constexpr int kMaxDevices = 64;
constexpr int kClasses = 5;          // single-array size classes (by rows of 512 B)
constexpr int kWidthGroups = 4;      // tune-table width groups: w <= 8, 16, 32, >= 64
constexpr int kStageBufs = 2;
constexpr size_t kStageChunk = size_t(64) << 20;   // host-path staging chunk (64 MiB)
constexpr uint64_t kMaxRowsPerWarp = uint64_t(1) << 26;  // u32 counters: 32 * 2^26 < 2^32

struct StreamTune {
  int variant;              // index into the stream kernel table
  int ctas_per_sm;          // blocks per SM (above the occupancy limit the grid runs in waves)
  uint32_t min_rows;        // fewest rows a warp should get before the grid grows
};
struct BatchTune {
  int variant;
  int ctas_per_sm;
  uint32_t item_rows[kBatchClasses];   // rows per work item, by array size class
  uint32_t grab;            // work items per atomic
};
struct RoofTune {
  int variant;
  int ctas_per_sm;
};
// Serving: one entry per request size class of the server (below 1 MiB,
// 16 MiB, 128 MiB, and above).
constexpr int kServeClasses = 4;
struct ServeTune {
  uint32_t light_rows;      // most work-item rows while the server is lightly loaded (0 = rows;
                            // items are then wave-aligned and at least half that long)
  uint32_t rows;            // work-item rows otherwise
  uint32_t streams;         // batch streams of the class that may run at once
  uint32_t cap;             // requests per batch
};
// Width group of w (1..256, a power of two): the tune table keeps one
// single-array entry per (width group, size class) and one batch entry per
// width group.
constexpr int width_group(int w) { return w <= 8 ? 0 : w == 16 ? 1 : w == 32 ? 2 : 3; }
constexpr int kGroupWidth[kWidthGroups] = {8, 16, 32, 64};   // the width each group is tuned at

struct TuneTable {
  StreamTune stream[kWidthGroups][kClasses];
  BatchTune batch[kWidthGroups];
  RoofTune roof;
  uint64_t max_rows_per_warp;   // single-array launch split (<= kMaxRowsPerWarp)
  uint32_t regroup;             // w = 8 short sequences: 1 = per-lane bit regroup, 0 = transpose
  uint32_t pdl;                 // 1 = launch with programmatic stream serialization
  uint32_t staged;              // selected counts of aligned spans: 0 = registers, k > 0 =
                                // bulk-copy staging with ring shape k - 1
  ServeTune serve[kServeClasses];
  uint64_t serve_light;         // in-flight input bytes below which the server counts as light
  uint32_t serve_strided;       // 1: serving work items take every K-th row of a request
  uint32_t serve_order;         // 0: a class's batch takes admitted requests in admission
                                // order; 1: smallest first
  uint32_t serve_promote_us;    // > 0: requests that have waited this long since they arrived
                                // may run on a free stream of the next smaller class
  int serve_shape;              // serving kernel's launch shape (index into the serve and
                                // batch families: block size, flush depth, load variant)
  uint32_t serve_mode;          // 0: size classes on prioritised streams; 1: dispatch by
                                // remaining bytes (read when a server is created)
  uint64_t srf_bytes;           // serve_mode 1: bytes of work items per launch, at most
  uint32_t srf_launches;        // serve_mode 1: launches in flight, at most
  uint32_t srf_rows;            // serve_mode 1: rows per work item
  uint32_t srf_class_rows[kServeClasses];   // serve_mode 1-3: rows per work item under
                                            // load by size class (0: srf_rows)
  uint32_t srf_age_us;          // serve_mode 1: a request waiting this long takes half a launch (0: off)
  uint32_t res_idle_us;         // serve_mode 3: the host stops the resident grid after this long idle
  uint32_t res_wait_us;         // serve_mode 3: the grid leaves after this long without a new run
  uint32_t multi_rows;          // pospopcnt_multi: most work-item rows (wave-aligned, at least 8)
  uint32_t multi_strided;       // pospopcnt_multi: 1 = items take every K-th row of their count
  long long wait_cycles;        // limit of a staged kernel's wait for a bulk copy (SM clock
                                // cycles, 0 .. kBulkWaitCycles; 0 = give up at once)
  char source[240];             // where the table came from (copied with the table: no heap)
  void set_source(const char *s);
};

// Scratch memory of one batched or gathered count: per-array prefix sums of
// work items (m + 1), the planning blocks' sums, the work counter and the
// device-side status word.
struct Scratch {
  uint64_t *item_start = nullptr;
  uint64_t *block_sum = nullptr;
  unsigned long long *next = nullptr;
  int *status = nullptr;
};

// Bytes of scratch for up to m_cap arrays, and its layout in a buffer of
// that size (256-byte aligned): item_start[m_cap + 1], one block sum per
// planning block (plus one), the work counter, the status word.
constexpr size_t scratch_bytes(size_t m_cap) {
  return 8 * (m_cap + 1) + 8 * ((m_cap + kPlanChunk - 1) / kPlanChunk + 1) + 16;
}
Scratch scratch_layout(void *buf, size_t m_cap);

struct Workspace {
  void *buf = nullptr;
  size_t m_cap = 0;
  Scratch scr;
  bool captured = false;   // used while the stream was being captured into a graph
};

struct Staging {
  bool ready = false;
  cudaStream_t copy = nullptr, comp = nullptr;
  void *buf[kStageBufs] = {nullptr, nullptr};
  cudaEvent_t copied[kStageBufs] = {nullptr, nullptr};
  cudaEvent_t consumed[kStageBufs] = {nullptr, nullptr};
  unsigned long long *dcounts = nullptr;
  unsigned long long *hcounts = nullptr;   // pinned, 256 entries
};

struct DevCtx {
  bool ready = false;
  int device = -1;
  int sms = 0;
  std::mutex mu;        // workspace map, tune table
  std::mutex host_mu;   // staging area
  std::unordered_map<cudaStream_t, Workspace> ws;
  std::vector<void *> retired;   // outgrown workspaces that a caller's graph may still use
  unsigned char *noalloc_scratch = nullptr;   // device address of the no-allocation array
  Staging st;
  TuneTable tune;
  int occ_stream[64] = {0};
  int occ_batch[64] = {0};
  int occ_roof[16] = {0};
  int occ_select_staged[16] = {0};
  int occ_serve[64] = {0};
  int occ_multi[64] = {0};
};

// Returns the context of the current device, setting it up if needed, or
// nullptr (rc set) on failure.
DevCtx *current_ctx(int *rc);
DevCtx *ctx_for_device(int device, int *rc);

int size_class(uint64_t rows);
TuneTable default_tune();
int find_variant(bool batch, int bs, int minb, int depth, int hint);
// Parses a tune table (text format in pospop_api.cu); on failure returns
// POSPOP_EINVAL and, if bad_line is not null, the 1-based failing line.
int parse_tune(const char *text, TuneTable *out, int *bad_line = nullptr);
std::string format_tune(const DevCtx &ctx, const TuneTable &t);

// Launch plan of one single-array count.
struct StreamPlan {
  int variant;
  unsigned grid;
  unsigned block;
  uint64_t rows;
  uint64_t rows_per_launch;
  int launches;
  int cls;
  int cps;
};
StreamPlan plan_stream(const DevCtx &ctx, const TuneTable &t, int w, uint64_t rows);

// Enqueue the single-array count of [bytes, bytes + nbytes) (device
// addressable) into counts (device, w entries) on `stream`.
int launch_stream_with(const DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                       const void *bytes, size_t nbytes, cudaStream_t stream);
int launch_stream(DevCtx &ctx, int w, unsigned long long *counts, const void *bytes,
                  size_t nbytes, cudaStream_t stream);
int launch_batch_with(DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                      const void *base, const uint64_t *offsets, size_t m, cudaStream_t stream);
// The batched count over CSR offsets with the given scratch (room for m
// arrays): clears the status word, then enqueues the three planning kernels
// and the persistent counting kernel on `stream`.  Every batched form (the
// per-stream workspace, a graph's own workspace, the no-allocation array)
// launches through this one routine.
int launch_batch_scratch(const DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                         const void *base, const uint64_t *offsets, size_t m,
                         const Scratch &scr, cudaStream_t stream);
// status: a device int the bulk-copy form sets to POSPOP_ETIMEDOUT when a
// staging wait expires (required for that form, ignored by the others);
// wait_cycles: that wait's limit.
int launch_roofline_with(const DevCtx &ctx, const RoofTune &rt, const void *bytes, size_t nbytes,
                         unsigned long long *sum, int *status, long long wait_cycles,
                         cudaStream_t stream, bool pdl);

// A pointer the device can read or write (device memory of ctx's device,
// managed memory, or pinned host memory mapped into the device's address
// space); *devptr receives the address to give a kernel.
bool device_addressable(const void *p, int device, const void **devptr);

// Serving kernel helpers (pospop_serve.cu), shared by the serving loop and
// the autotuner.  Rows of 512 B of the byte span [ptr, ptr + nbytes):
uint64_t serve_rows(const void *ptr, uint64_t nbytes);
// Light-load work-item rows of a batch of `rows` rows: at most `most`, at
// least `least` (0: half of `most`, at least 8), the number of items a whole
// multiple of the resident warps of serve variant `variant` where the batch
// is large enough.
uint32_t serve_light_rows(const DevCtx &ctx, int variant, uint64_t rows, uint32_t most,
                          uint32_t least = 0);
// Launch serve variant v on the planned parameter block P (nothing if P
// has no work items).
int serve_launch(int shape, const ServeParams &P, cudaStream_t stream);

// Device address of the no-allocation batch's scratch array on the current
// device (pospop_noalloc.cu); called once per device when its context is
// set up, with that device current.
int noalloc_lookup(unsigned char **out);

void note_launches(uint64_t n);

// cudaLaunchKernel, or with pdl set, the same launch with programmatic stream
// serialization (the kernel waits for its predecessor in pdl_enter()).
cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, void **args, cudaStream_t stream,
                          bool pdl, size_t smem = 0);

}  // namespace pospop

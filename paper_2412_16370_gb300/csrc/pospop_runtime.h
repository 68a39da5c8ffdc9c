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
  uint32_t item_rows;       // rows per work item
  uint32_t grab;            // work items per atomic
};
struct RoofTune {
  int variant;
  int ctas_per_sm;
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
  char source[240];             // where the table came from (copied with the table: no heap)
  void set_source(const char *s);
};

struct Workspace {
  void *buf = nullptr;
  size_t m_cap = 0;
  uint64_t *item_start = nullptr;
  uint64_t *block_sum = nullptr;
  unsigned long long *next = nullptr;
  int *status = nullptr;
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
  Staging st;
  TuneTable tune;
  int occ_stream[64] = {0};
  int occ_batch[64] = {0};
  int occ_roof[16] = {0};
  int occ_select_staged[16] = {0};
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
// status: a device int the bulk-copy form sets to POSPOP_ETIMEDOUT when a
// staging wait expires (required for that form, ignored by the others).
int launch_roofline_with(const DevCtx &ctx, const RoofTune &rt, const void *bytes, size_t nbytes,
                         unsigned long long *sum, int *status, cudaStream_t stream, bool pdl);

void note_launches(uint64_t n);

// cudaLaunchKernel, or with pdl set, the same launch with programmatic stream
// serialization (the kernel waits for its predecessor in pdl_enter()).
cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, void **args, cudaStream_t stream,
                          bool pdl, size_t smem = 0);

}  // namespace pospop

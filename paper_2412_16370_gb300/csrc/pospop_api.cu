// pospop_api.cu -- the C ABI of libpospopcnt.so (declared in
// include/pospopcnt.h): argument checks, per-device contexts, workspaces,
// launch planning, the host-memory path and CUDA graphs.
//
// Every count runs in the sm_103a kernels (pospop_stream.cu, pospop_batch.cu,
// pospop_gather.cu, pospop_select.cu, pospop_roofline.cu); this file only
// validates, plans and enqueues.
#include <dlfcn.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pospopcnt.h"
#include "pospop_runtime.h"

namespace pospop {

static std::mutex g_mu;
static DevCtx *g_ctx[kMaxDevices] = {nullptr};
static std::atomic<uint64_t> g_launches{0};

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static bool valid_w(int w) {
  return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64;
}

// The single-array, batched and gathered forms also take the wider folds.
static bool valid_w_single(int w) { return valid_w(w) || w == 128 || w == 256; }
static bool valid_w_multi(int w) { return valid_w_single(w); }

// Index in a kernel family (stride `step`) of the variant launched with the
// same block shape as `want` -- a kernel must be launched with the block size
// it was compiled for -- preferring the same load hint.  -1 if none.
static int pick_shape(int count, const Variant &(*get)(int), int step, const Variant &want) {
  int same_shape = -1;
  for (int i = 0; i < count; i += step) {
    const Variant &c = get(i);
    if (c.bs != want.bs || c.minb != want.minb) continue;
    if (c.hint == want.hint) return i;
    if (same_shape < 0) same_shape = i;
  }
  return same_shape;
}

// ---------------------------------------------------------------------------
// Tune table.
// ---------------------------------------------------------------------------
void TuneTable::set_source(const char *s) { snprintf(source, sizeof source, "%s", s ? s : ""); }

int size_class(uint64_t rows) {
  if (rows <= 64) return 0;          // <= 32 KiB
  if (rows <= 2048) return 1;        // <= 1 MiB
  if (rows <= 65536) return 2;       // <= 32 MiB
  if (rows <= (1u << 21)) return 3;  // <= 1 GiB
  return 4;
}

int find_variant(bool batch, int bs, int minb, int depth, int hint) {
  const int n = batch ? batch_variant_count() : stream_variant_count();
  for (int i = 0; i < n; i++) {
    const Variant &v = batch ? batch_variant(i) : stream_variant(i);
    if (v.bs == bs && v.minb == minb && v.depth == depth && v.hint == hint) return i;
  }
  return -1;
}

static int find_roof_variant(int bs, int hint) {
  for (int i = 0; i < roofline_variant_count(); i++)
    if (roofline_variant(i).bs == bs && roofline_variant(i).hint == hint) return i;
  return -1;
}

TuneTable default_tune() {
  TuneTable t;
  const int sv = find_variant(false, 512, 1, 16, 1);
  const uint32_t minrows[kClasses] = {2, 4, 8, 16, 16};
  for (int g = 0; g < kWidthGroups; g++) {
    for (int c = 0; c < kClasses; c++) t.stream[g][c] = StreamTune{sv, 1, minrows[c]};
    t.batch[g] = BatchTune{find_variant(true, 256, 2, 16, 1), 2, {511, 511, 511, 511}, 1};
  }
  t.roof = RoofTune{find_roof_variant(512, 1), 4};
  t.max_rows_per_warp = kMaxRowsPerWarp;
  t.regroup = 0;
  t.pdl = 1;
  t.staged = 3;   // 16 warps x 1 stage: measured fastest on GB300
  t.wait_cycles = kBulkWaitCycles;
  // serving (measured on GB300, Poisson traces at 0.3 / 0.6 / 0.9 of the
  // large-array rate): longer items for the larger classes under load, short
  // wave-aligned items while lightly loaded; the largest class one request
  // a batch, the smallest waiting request first
  t.serve[0] = ServeTune{8, 127, 64, 1024};
  t.serve[1] = ServeTune{32, 255, 64, 1024};
  t.serve[2] = ServeTune{127, 511, 64, 1024};
  t.serve[3] = ServeTune{0, 511, 64, 1};
  t.serve_light = uint64_t(512) << 20;
  t.serve_strided = 0;
  t.serve_order = 1;
  t.serve_promote_us = 0;
  // load variant 0 (the variant-1 serving kernels keep part of their state
  // in local memory, 80-88 bytes a thread) and flush depth 32 (measured on
  // GB300: 0.9-load p99 367-370 us against 395-397 us at depth 16)
  t.serve_shape = find_variant(true, 512, 1, 32, 0);
  // dispatch by remaining bytes, 128 MiB of work items a launch, five
  // launches in flight (measured on GB300 with a Poisson trace at 0.9 load:
  // p99 238-239 us against 271-284 us with four launches and 366-370 us
  // for the size classes, and the same latency for a lone request)
  t.serve_mode = 1;
  t.srf_bytes = uint64_t(128) << 20;
  t.srf_launches = 5;
  t.srf_rows = 255;
  // under load, 15- and 127-row items for requests below 1 MiB and 16 MiB
  // (measured on GB300 with five launches: 0.9-load p50 49 against 62 us,
  // p99 241-243 against 245-253 us)
  t.srf_class_rows[0] = 15;
  t.srf_class_rows[1] = 127;
  t.srf_class_rows[2] = 0;
  t.srf_class_rows[3] = 0;
  t.srf_age_us = 0;
  t.res_idle_us = 2000;
  t.res_wait_us = 200000;
  t.multi_rows = 1024;
  t.multi_strided = 1;
  t.set_source("built-in defaults");
  return t;
}

// Text format, one entry per line ('#' starts a comment):
//   stream [<w>] <class> <bs> <minb> <depth> <hint> <ctas_per_sm> <min_rows>
//   batch [<w>] <bs> <minb> <depth> <hint> <ctas_per_sm> <item_rows> <grab>
//                                 (<w> in {8, 16, 32, 64} sets the entry of that
//                                  width group: 8 stands for w <= 8, 64 for
//                                  w >= 64; without it the entry is every group's;
//                                  item_rows is every array size class's)
//   batch_rows [<w>] <r0> <r1> <r2> <r3>
//                                 (work-item rows of arrays of at most 2 KiB, 32 KiB,
//                                  1 MiB, and above, 1 .. 2^20; after the batch line
//                                  of the same width groups)
//   roofline <bs> <hint> <ctas_per_sm>
//   split <max_rows_per_warp>     (1 .. 2^26; a single-array count is split into
//                                  several launches so that no warp takes more)
//   short <0|1>                   (w = 8 sequences of <= 3 rows: 0 = transpose
//                                  flush, 1 = per-lane bit regroup)
//   pdl <0|1>                     (1 = programmatic dependent launch: a kernel's
//                                  launch overlaps the previous kernel's run)
//   staged <0|k>                  (k > 0: selected counts of 16-byte-aligned spans
//                                  stage their input in shared memory by bulk copies,
//                                  ring shape k: 1 = 8 warps x 3 stages, 2 = 12 x 2,
//                                  3 = 16 x 1; 0 = loads into registers)
//   serve <class> <light_rows> <rows> <streams> <cap>
//                                 (serving size class 0..3 = below 1 MiB, 16 MiB,
//                                  128 MiB, above: most work-item rows while lightly
//                                  loaded (0 = rows; items are wave-aligned, at least
//                                  half that) and rows otherwise (1 .. 2^20), batch
//                                  streams of the class running at once (1 .. 64),
//                                  requests per batch (1 .. 1024))
//   serve_light <bytes>           (in-flight input bytes below which the server counts
//                                  as lightly loaded)
//   serve_strided <0|1>           (1: a serving work item of a request of K items
//                                  counts every K-th row; 0: a contiguous run)
//   serve_order <0|1>             (a class's next batch takes its admitted requests in
//                                  admission order (0) or smallest first (1))
//   serve_shape <bs> <minb> <depth> <hint>
//                                 (the serving kernel's launch shape)
//   serve_mode <0|1|2|3>          (read when a server is created: 0 = size classes on
//                                  prioritised streams; 1 = dispatch by remaining bytes;
//                                  2 = the same per size class of the bytes left, on the
//                                  classes' prioritised streams; 3 = smallest remaining
//                                  first through a device-side queue into one resident
//                                  grid, serve_srf's <bytes> the queue's unclaimed work)
//   serve_srf_class <r0> <r1> <r2> <r3>
//                                 (serve_mode 1-3: rows per work item under load for
//                                  requests of size class 0 .. 3, 0 .. 2^20; 0 takes
//                                  serve_srf's rows)
//   serve_srf_age <us>            (serve_mode 1: 0 = off; else the longest-waiting
//                                  request that has waited this long since it arrived
//                                  takes up to half of the next launch, 1 .. 10^7)
//   serve_resident <idle_us> <wait_us>
//                                 (serve_mode 3: the host stops the resident grid after
//                                  idle_us without work; the grid leaves by itself after
//                                  wait_us without a new run; 1 .. 10^7 each)
//   serve_srf <bytes> <launches> <rows>
//                                 (serve_mode 1 and 2: work-item bytes per launch, at
//                                  least one item; launches in flight (per class with
//                                  mode 2), 1 .. 64; rows per item under load, 1 .. 2^20,
//                                  or 0 for the `serve` entry's rows of the request's
//                                  class; the bytes at least 512 x the rows)
//   serve_promote <us>            (0 = off; else requests of a class that have waited
//                                  this long since they arrived may run as a batch on a
//                                  free stream of the next smaller class, 1 .. 10^7)
//   multi <rows> <0|1>            (pospopcnt_multi: most work-item rows, 8 .. 2^20,
//                                  and 1 = items take every K-th row of their count)
//   wait <cycles>                 (0 .. 2^31: how long a staged kernel waits for a
//                                  stage's bulk copy, in SM clock cycles, before it
//                                  reports POSPOP_ETIMEDOUT and leaves; default 2^31,
//                                  about a second; 0 gives up at once, which tests
//                                  the time-out exit on healthy copies)
// The integers after the line's keyword, at most max of them: their number,
// or -1 for a token that is not an integer or one too many.
static int read_ints(const std::string &line, long long *v, int max) {
  const char *q = line.c_str();
  while (*q == ' ' || *q == '\t') q++;
  while (*q && *q != ' ' && *q != '\t') q++;   // the keyword
  int n = 0;
  while (true) {
    while (*q == ' ' || *q == '\t' || *q == '\r') q++;
    if (!*q) return n;
    if (n == max) return -1;
    char *end = nullptr;
    v[n] = strtoll(q, &end, 10);
    if (end == q) return -1;
    n++;
    q = end;
  }
}

// Width groups named by an optional leading <w>: [first, last) of the groups.
static bool tune_groups(long long w, bool given, int *first, int *last) {
  if (!given) {
    *first = 0;
    *last = kWidthGroups;
    return true;
  }
  for (int g = 0; g < kWidthGroups; g++)
    if (w == kGroupWidth[g]) {
      *first = g;
      *last = g + 1;
      return true;
    }
  return false;
}

int parse_tune(const char *text, TuneTable *out, int *bad_line) {
  TuneTable t = default_tune();
  std::string s(text);
  size_t pos = 0;
  int lineno = 0;
  while (pos < s.size()) {
    size_t nl = s.find('\n', pos);
    if (nl == std::string::npos) nl = s.size();
    std::string line = s.substr(pos, nl - pos);
    pos = nl + 1;
    lineno++;
    if (bad_line) *bad_line = lineno;   // the line being read, if it fails
    const size_t hash = line.find('#');
    if (hash != std::string::npos) line.resize(hash);
    char kind[16] = {0};
    if (sscanf(line.c_str(), "%15s", kind) != 1) continue;
    // every field is a decimal integer; a line with a stray token or the
    // wrong number of fields is refused
    long long a[8];
    const int n = read_ints(line, a, 8);
    const bool is_stream = strcmp(kind, "stream") == 0;
    if (is_stream || strcmp(kind, "batch") == 0) {
      int g0 = 0, g1 = 0;
      if ((n != 7 && n != 8) || !tune_groups(a[0], n == 8, &g0, &g1)) return POSPOP_EINVAL;
      const long long *f = a + (n - 7);   // the seven fields after the optional <w>
      for (int i = 0; i < 7; i++)
        if (f[i] < 0 || f[i] > (1ll << 30)) return POSPOP_EINVAL;
      if (is_stream) {
        const int c = (int)f[0], v = find_variant(false, (int)f[1], (int)f[2], (int)f[3], (int)f[4]);
        if (c >= kClasses || v < 0 || f[5] < 1 || f[6] < 1) return POSPOP_EINVAL;
        for (int g = g0; g < g1; g++) t.stream[g][c] = StreamTune{v, (int)f[5], (uint32_t)f[6]};
      } else {
        const int v = find_variant(true, (int)f[0], (int)f[1], (int)f[2], (int)f[3]);
        if (v < 0 || f[4] < 1 || f[5] < 1 || f[5] > (1 << 20) || f[6] < 1 || f[6] > 64)
          return POSPOP_EINVAL;
        const uint32_t ir = (uint32_t)f[5];
        for (int g = g0; g < g1; g++)
          t.batch[g] = BatchTune{v, (int)f[4], {ir, ir, ir, ir}, (uint32_t)f[6]};
      }
    } else if (strcmp(kind, "batch_rows") == 0) {
      int g0 = 0, g1 = 0;
      if ((n != kBatchClasses && n != kBatchClasses + 1) ||
          !tune_groups(a[0], n == kBatchClasses + 1, &g0, &g1))
        return POSPOP_EINVAL;
      const long long *f = a + (n - kBatchClasses);
      for (int c = 0; c < kBatchClasses; c++)
        if (f[c] < 1 || f[c] > (1 << 20)) return POSPOP_EINVAL;
      for (int g = g0; g < g1; g++)
        for (int c = 0; c < kBatchClasses; c++) t.batch[g].item_rows[c] = (uint32_t)f[c];
    } else if (strcmp(kind, "short") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 1) return POSPOP_EINVAL;
      t.regroup = (uint32_t)a[0];
    } else if (strcmp(kind, "pdl") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 1) return POSPOP_EINVAL;
      t.pdl = (uint32_t)a[0];
    } else if (strcmp(kind, "staged") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > select_staged_variant_count() / 4) return POSPOP_EINVAL;
      t.staged = (uint32_t)a[0];
    } else if (strcmp(kind, "serve") == 0) {
      if (n != 5 || a[0] < 0 || a[0] >= kServeClasses || a[1] < 0 || a[1] > (1 << 20) ||
          a[2] < 1 || a[2] > (1 << 20) || a[3] < 1 || a[3] > 64 || a[4] < 1 || a[4] > 1024)
        return POSPOP_EINVAL;
      t.serve[a[0]] = ServeTune{(uint32_t)a[1], (uint32_t)a[2], (uint32_t)a[3], (uint32_t)a[4]};
    } else if (strcmp(kind, "serve_light") == 0) {
      if (n != 1 || a[0] < 0) return POSPOP_EINVAL;
      t.serve_light = (uint64_t)a[0];
    } else if (strcmp(kind, "serve_strided") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 1) return POSPOP_EINVAL;
      t.serve_strided = (uint32_t)a[0];
    } else if (strcmp(kind, "serve_mode") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 3) return POSPOP_EINVAL;
      t.serve_mode = (uint32_t)a[0];
    } else if (strcmp(kind, "serve_srf") == 0) {
      if (n != 3 || a[2] < 0 || a[2] > (1 << 20) || a[1] < 1 || a[1] > 64 ||
          a[0] < 512 * std::max<long long>(a[2], 1))
        return POSPOP_EINVAL;
      t.srf_bytes = (uint64_t)a[0];
      t.srf_launches = (uint32_t)a[1];
      t.srf_rows = (uint32_t)a[2];
    } else if (strcmp(kind, "serve_srf_class") == 0) {
      if (n != kServeClasses) return POSPOP_EINVAL;
      for (int k = 0; k < kServeClasses; k++)
        if (a[k] < 0 || a[k] > (1 << 20)) return POSPOP_EINVAL;
      for (int k = 0; k < kServeClasses; k++) t.srf_class_rows[k] = (uint32_t)a[k];
    } else if (strcmp(kind, "serve_srf_age") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 10000000) return POSPOP_EINVAL;
      t.srf_age_us = (uint32_t)a[0];
    } else if (strcmp(kind, "serve_resident") == 0) {
      if (n != 2 || a[0] < 1 || a[0] > 10000000 || a[1] < 1 || a[1] > 10000000)
        return POSPOP_EINVAL;
      t.res_idle_us = (uint32_t)a[0];
      t.res_wait_us = (uint32_t)a[1];
    } else if (strcmp(kind, "serve_shape") == 0) {
      if (n != 4) return POSPOP_EINVAL;
      const int v = find_variant(true, (int)a[0], (int)a[1], (int)a[2], (int)a[3]);
      if (v < 0) return POSPOP_EINVAL;
      t.serve_shape = v;
    } else if (strcmp(kind, "serve_promote") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 10000000) return POSPOP_EINVAL;
      t.serve_promote_us = (uint32_t)a[0];
    } else if (strcmp(kind, "serve_order") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > 1) return POSPOP_EINVAL;
      t.serve_order = (uint32_t)a[0];
    } else if (strcmp(kind, "multi") == 0) {
      if (n != 2 || a[0] < 8 || a[0] > (1 << 20) || a[1] < 0 || a[1] > 1) return POSPOP_EINVAL;
      t.multi_rows = (uint32_t)a[0];
      t.multi_strided = (uint32_t)a[1];
    } else if (strcmp(kind, "wait") == 0) {
      if (n != 1 || a[0] < 0 || a[0] > kBulkWaitCycles) return POSPOP_EINVAL;
      t.wait_cycles = a[0];
    } else if (strcmp(kind, "split") == 0) {
      if (n != 1 || a[0] < 1 || (unsigned long long)a[0] > kMaxRowsPerWarp) return POSPOP_EINVAL;
      t.max_rows_per_warp = (uint64_t)a[0];
    } else if (strcmp(kind, "roofline") == 0) {
      if (n != 3 || a[0] < 1 || a[0] > 1024 || a[1] < 0 || a[1] > 16 || a[2] < 1 ||
          a[2] > 1024)
        return POSPOP_EINVAL;
      const int v = find_roof_variant((int)a[0], (int)a[1]);
      if (v < 0) return POSPOP_EINVAL;
      t.roof = RoofTune{v, (int)a[2]};
    } else {
      return POSPOP_EINVAL;
    }
  }
  if (bad_line) *bad_line = 0;
  *out = t;
  return POSPOP_OK;
}

std::string format_tune(const DevCtx &ctx, const TuneTable &t) {
  std::string s;
  char line[256];
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx.device) != cudaSuccess) {
    cudaGetLastError();
    snprintf(prop.name, sizeof(prop.name), "unknown");
  }
  s += std::string("# pospopcnt tune table: ") + prop.name + ", " + std::to_string(ctx.sms) +
       " SMs (" + t.source + ")\n";
  // an entry that is the same for every width group is written once,
  // without <w>
  s += "# stream [<w>] <class> <bs> <minb> <depth> <hint> <ctas_per_sm> <min_rows>\n";
  for (int c = 0; c < kClasses; c++) {
    bool same = true;
    for (int g = 1; g < kWidthGroups; g++) {
      const StreamTune &a = t.stream[0][c], &b = t.stream[g][c];
      same = same && a.variant == b.variant && a.ctas_per_sm == b.ctas_per_sm &&
             a.min_rows == b.min_rows;
    }
    for (int g = 0; g < (same ? 1 : kWidthGroups); g++) {
      const StreamTune &e = t.stream[g][c];
      const Variant &v = stream_variant(e.variant);
      char wfield[16] = "";
      if (!same) snprintf(wfield, sizeof wfield, "%d ", kGroupWidth[g]);
      snprintf(line, sizeof line, "stream %s%d %d %d %d %d %d %u\n", wfield, c, v.bs, v.minb,
               v.depth, v.hint, e.ctas_per_sm, e.min_rows);
      s += line;
    }
  }
  {
    s += "# batch [<w>] <bs> <minb> <depth> <hint> <ctas_per_sm> <item_rows> <grab>\n";
    s += "# batch_rows [<w>] <rows: arrays <= 2 KiB> <<= 32 KiB> <<= 1 MiB> <above>>\n";
    bool same = true;
    for (int g = 1; g < kWidthGroups; g++) {
      const BatchTune &a = t.batch[0], &b = t.batch[g];
      same = same && a.variant == b.variant && a.ctas_per_sm == b.ctas_per_sm &&
             a.grab == b.grab;
      for (int c = 0; c < kBatchClasses; c++) same = same && a.item_rows[c] == b.item_rows[c];
    }
    for (int g = 0; g < (same ? 1 : kWidthGroups); g++) {
      const BatchTune &e = t.batch[g];
      const Variant &v = batch_variant(e.variant);
      char wfield[16] = "";
      if (!same) snprintf(wfield, sizeof wfield, "%d ", kGroupWidth[g]);
      snprintf(line, sizeof line, "batch %s%d %d %d %d %d %u %u\n", wfield, v.bs, v.minb, v.depth,
               v.hint, e.ctas_per_sm, e.item_rows[kBatchClasses - 1], e.grab);
      s += line;
      bool uniform = true;
      for (int c = 0; c < kBatchClasses; c++) uniform = uniform && e.item_rows[c] == e.item_rows[0];
      if (!uniform) {
        snprintf(line, sizeof line, "batch_rows %s%u %u %u %u\n", wfield, e.item_rows[0],
                 e.item_rows[1], e.item_rows[2], e.item_rows[3]);
        s += line;
      }
    }
  }
  snprintf(line, sizeof line, "# short <0 transpose | 1 per-lane regroup> (w = 8, <= 3 rows)\nshort %u\n",
           t.regroup);
  s += line;
  snprintf(line, sizeof line, "# pdl <0 | 1 programmatic dependent launch>\npdl %u\n", t.pdl);
  s += line;
  snprintf(line, sizeof line,
           "# staged <0 registers | k bulk-copy staging ring shape> (selected counts)\nstaged %u\n",
           t.staged);
  s += line;
  if (t.max_rows_per_warp != kMaxRowsPerWarp) {
    snprintf(line, sizeof line, "split %llu\n", (unsigned long long)t.max_rows_per_warp);
    s += line;
  }
  s += "# serve <class> <light_rows> <rows> <streams> <cap>\n";
  for (int k = 0; k < kServeClasses; k++) {
    const ServeTune &e = t.serve[k];
    snprintf(line, sizeof line, "serve %d %u %u %u %u\n", k, e.light_rows, e.rows, e.streams,
             e.cap);
    s += line;
  }
  snprintf(line, sizeof line,
           "serve_light %llu\nserve_strided %u\nserve_order %u\nserve_promote %u\n",
           (unsigned long long)t.serve_light, t.serve_strided, t.serve_order,
           t.serve_promote_us);
  s += line;
  {
    const Variant &v = serve_variant(t.serve_shape);
    snprintf(line, sizeof line,
             "serve_shape %d %d %d %d\nserve_mode %u\nserve_srf %llu %u %u\n"
             "serve_srf_class %u %u %u %u\nserve_srf_age %u\nserve_resident %u %u\n",
             v.bs, v.minb, v.depth, v.hint, t.serve_mode, (unsigned long long)t.srf_bytes,
             t.srf_launches, t.srf_rows, t.srf_class_rows[0], t.srf_class_rows[1],
             t.srf_class_rows[2], t.srf_class_rows[3], t.srf_age_us, t.res_idle_us, t.res_wait_us);
    s += line;
  }
  snprintf(line, sizeof line, "# multi <most item rows> <0 contiguous | 1 strided items>\nmulti %u %u\n",
           t.multi_rows, t.multi_strided);
  s += line;
  if (t.wait_cycles != kBulkWaitCycles) {
    snprintf(line, sizeof line, "wait %lld\n", t.wait_cycles);
    s += line;
  }
  {
    const Variant &v = roofline_variant(t.roof.variant);
    s += "# roofline <bs> <hint> <ctas_per_sm>\n";
    snprintf(line, sizeof line, "roofline %d %d %d\n", v.bs, v.hint, t.roof.ctas_per_sm);
    s += line;
  }
  return s;
}

static bool read_file(const std::string &path, std::string *out) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::string s;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
  fclose(f);
  *out = s;
  return true;
}

// The tune table installed at set-up: $POSPOP_TUNE_FILE, else
// pospopcnt_tune.txt next to this shared library, else the defaults.
static TuneTable initial_tune() {
  std::string path;
  if (const char *env = getenv("POSPOP_TUNE_FILE")) {
    path = env;
  } else {
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&initial_tune), &info) && info.dli_fname) {
      std::string so = info.dli_fname;
      const size_t slash = so.rfind('/');
      path = (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) +
             "/pospopcnt_tune.txt";
    }
  }
  std::string text;
  TuneTable t;
  if (!path.empty() && read_file(path, &text) && parse_tune(text.c_str(), &t) == POSPOP_OK) {
    t.set_source(path.c_str());
    return t;
  }
  return default_tune();
}

// ---------------------------------------------------------------------------
// Device contexts.
// ---------------------------------------------------------------------------
static int init_ctx(DevCtx &c, int device) {
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return POSPOP_ECUDA; }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  for (int i = 0; i < stream_variant_count(); i++) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_variant(i).fn,
                                                      stream_variant(i).bs, 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    c.occ_stream[i] = n > 0 ? n : 1;
  }
  for (int i = 0; i < batch_variant_count(); i++) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_variant(i).fn,
                                                      batch_variant(i).bs, 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    c.occ_batch[i] = n > 0 ? n : 1;
  }
  for (int i = 0; i < serve_variant_count(); i++) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, serve_variant(i).fn,
                                                      serve_variant(i).bs, 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    c.occ_serve[i] = n > 0 ? n : 1;
  }
  for (int i = 0; i < multi_variant_count(); i++) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, multi_variant(i).fn,
                                                      multi_variant(i).bs, 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    c.occ_multi[i] = n > 0 ? n : 1;
  }
  for (int i = 0; i < roofline_variant_count(); i++) {
    const Variant &v = roofline_variant(i);
    int n = 0;
    if ((v.smem > 0 && cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            v.smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, v.bs, (size_t)v.smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    c.occ_roof[i] = n > 0 ? n : 1;
  }
  for (int i = 0; i < select_staged_variant_count(); i++) {
    const Variant &v = select_staged_variant(i);
    int n = 0;
    if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, v.bs, (size_t)v.smem) !=
            cudaSuccess) {
      cudaGetLastError();
      n = 0;   // the staged form is then not used
    }
    c.occ_select_staged[i] = n;
  }
  // the no-allocation batch's scratch array: its device address, looked up
  // once per device with that device current
  if (noalloc_lookup(&c.noalloc_scratch) != POSPOP_OK) return POSPOP_ECUDA;
  c.device = device;
  c.sms = sms;
  c.tune = initial_tune();
  c.ready = true;
  return POSPOP_OK;
}

DevCtx *ctx_for_device(int device, int *rc) {
  if (device < 0 || device >= kMaxDevices) { *rc = POSPOP_EINVAL; return nullptr; }
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_ctx[device]) g_ctx[device] = new DevCtx();
  DevCtx *c = g_ctx[device];
  if (!c->ready) {
    *rc = init_ctx(*c, device);
    if (*rc != POSPOP_OK) return nullptr;
  }
  *rc = POSPOP_OK;
  return c;
}

DevCtx *current_ctx(int *rc) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    *rc = POSPOP_ECUDA;
    return nullptr;
  }
  return ctx_for_device(dev, rc);
}

static void free_staging(Staging &st) {
  for (int b = 0; b < kStageBufs; b++) {
    if (st.buf[b]) cudaFree(st.buf[b]);
    if (st.copied[b]) cudaEventDestroy(st.copied[b]);
    if (st.consumed[b]) cudaEventDestroy(st.consumed[b]);
  }
  if (st.dcounts) cudaFree(st.dcounts);
  if (st.hcounts) cudaFreeHost(st.hcounts);
  if (st.copy) cudaStreamDestroy(st.copy);
  if (st.comp) cudaStreamDestroy(st.comp);
  st = Staging();
  cudaGetLastError();
}

static void free_ctx(DevCtx &c) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(c.device);
  cudaDeviceSynchronize();
  for (auto &kv : c.ws)
    if (kv.second.buf) cudaFree(kv.second.buf);
  c.ws.clear();
  for (void *b : c.retired) cudaFree(b);
  c.retired.clear();
  free_staging(c.st);
  c.ready = false;
  cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
}

// ---------------------------------------------------------------------------
// Pointer kinds.
// ---------------------------------------------------------------------------
enum PtrKind { kDev, kPinned, kPageable, kBadPtr };

static PtrKind classify(const void *p, int device, const void **devptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kBadPtr;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      if (a.device != device) return kBadPtr;
      if (devptr) *devptr = p;
      return kDev;
    case cudaMemoryTypeManaged:
      if (devptr) *devptr = p;
      return kDev;
    case cudaMemoryTypeHost:
      if (!a.devicePointer) return kBadPtr;
      if (devptr) *devptr = a.devicePointer;
      return kPinned;
    default:
      return kPageable;
  }
}

bool device_addressable(const void *p, int device, const void **devptr) {
  const PtrKind k = classify(p, device, devptr);
  return k == kDev || k == kPinned;
}

// ---------------------------------------------------------------------------
// Kernel launch, optionally as a programmatic dependent launch.
// ---------------------------------------------------------------------------
cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, void **args, cudaStream_t stream,
                          bool pdl, size_t smem) {
  if (!pdl) return cudaLaunchKernel(fn, grid, block, args, smem, stream);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1] = {};
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------------------
// Single-array launches.
// ---------------------------------------------------------------------------
StreamPlan plan_stream(const DevCtx &ctx, const TuneTable &t, int w, uint64_t rows) {
  StreamPlan p;
  p.cls = size_class(rows);
  const StreamTune &st = t.stream[width_group(w)][p.cls];
  p.variant = st.variant;
  const Variant &v = stream_variant(st.variant);
  // ctas_per_sm above the occupancy limit is allowed: the grid then runs in
  // waves (measured on GB300: 2-4 waves of the grid-stride row schedule read
  // about 1% faster than one)
  int cps = st.ctas_per_sm;
  if (cps < 1) cps = 1;
  p.cps = cps;
  const uint64_t wpb = (uint64_t)v.bs / 32;
  const uint64_t max_grid = (uint64_t)ctx.sms * (uint64_t)cps;
  const uint64_t want_warps = (rows + st.min_rows - 1) / st.min_rows;
  uint64_t grid = (want_warps + wpb - 1) / wpb;
  if (grid < 1) grid = 1;
  if (grid > max_grid) grid = max_grid;
  p.grid = (unsigned)grid;
  p.block = (unsigned)v.bs;
  p.rows = rows;
  p.rows_per_launch = grid * wpb * t.max_rows_per_warp;
  p.launches = rows == 0 ? 0 : (int)((rows + p.rows_per_launch - 1) / p.rows_per_launch);
  return p;
}

int launch_stream_with(const DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                       const void *bytes, size_t nbytes, cudaStream_t stream) {
  if (nbytes == 0) return POSPOP_OK;
  const uint64_t p0 = (uint64_t)bytes, e = p0 + nbytes;
  StreamParams P;
  const uint64_t A = p0 & ~15ull;
  P.s.A = reinterpret_cast<const uint8_t *>(A);
  P.s.head = (uint32_t)(p0 - A);
  P.s.G = (((e + 15u) & ~15ull) - A) >> 4;
  P.s.tail = (uint32_t)(e - (A + 16u * (P.s.G - 1)));
  P.counts = counts;
  P.w = w;
  P.rot = (8u * P.s.head) & (uint32_t)(w - 1);
  P.regroup = t.regroup;
  const uint64_t R = (P.s.G + 31) >> 5;
  const StreamPlan pl = plan_stream(ctx, t, w, R);
  const Variant *vp = &stream_variant(pl.variant);
  if (w == 256) {   // the two-parity kernel with the planned block shape
    const int pick = pick_shape(stream256_variant_count(), stream256_variant, 1, *vp);
    if (pick < 0) return POSPOP_EINVAL;
    vp = &stream256_variant(pick);
  }
  const Variant &v = *vp;
  for (uint64_t rb = 0; rb < R; rb += pl.rows_per_launch) {
    P.row_begin = rb;
    P.row_end = (R - rb > pl.rows_per_launch) ? rb + pl.rows_per_launch : R;
    void *args[] = {&P};
    if (launch_kernel(v.fn, dim3(pl.grid), dim3(pl.block), args, stream, t.pdl != 0) !=
        cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    note_launches(1);
  }
  return POSPOP_OK;
}

int launch_stream(DevCtx &ctx, int w, unsigned long long *counts, const void *bytes, size_t nbytes,
                  cudaStream_t stream) {
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(ctx.mu);
    t = ctx.tune;
  }
  return launch_stream_with(ctx, t, w, counts, bytes, nbytes, stream);
}

int launch_roofline_with(const DevCtx &ctx, const RoofTune &rt, const void *bytes, size_t nbytes,
                         unsigned long long *sum, int *status, long long wait_cycles,
                         cudaStream_t stream, bool pdl) {
  const uint64_t p0 = (uint64_t)bytes;
  const uint64_t A = (p0 + 15u) & ~15ull, E = (p0 + nbytes) & ~15ull;
  if (E <= A) return POSPOP_OK;
  RooflineParams P;
  P.A = reinterpret_cast<const uint8_t *>(A);
  P.G = (E - A) >> 4;
  P.sum = sum;
  P.status = status;
  P.wait_cycles = wait_cycles;
  const Variant &v = roofline_variant(rt.variant);
  if (v.smem > 0 && !status) return POSPOP_EINVAL;
  int cps = rt.ctas_per_sm;   // above the occupancy limit: waves, as for the count
  if (cps < 1) cps = 1;
  // a warp's unit of work: a row of 32 granules (direct loads) or a chunk of
  // 512 granules (bulk-copy staging)
  const uint64_t units = v.smem > 0 ? (P.G + 511) >> 9 : (P.G + 31) >> 5;
  uint64_t grid = (units + (v.bs / 32) - 1) / (v.bs / 32);
  uint64_t max_grid = (uint64_t)ctx.sms * cps;
  // an input too small to give every warp of that grid 32 units runs in one
  // wave of resident blocks instead (the waves pay only for large inputs)
  const uint64_t wave = (uint64_t)ctx.sms * (uint64_t)std::max(1, ctx.occ_roof[rt.variant]);
  if (max_grid > wave && units < max_grid * (v.bs / 32) * 32) max_grid = wave;
  if (grid > max_grid) grid = max_grid;
  if (grid < 1) grid = 1;
  void *args[] = {&P};
  if (launch_kernel(v.fn, dim3((unsigned)grid), dim3(v.bs), args, stream, pdl, (size_t)v.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(1);
  return POSPOP_OK;
}

// ---------------------------------------------------------------------------
// Batched launches and their workspace.
// ---------------------------------------------------------------------------
Scratch scratch_layout(void *buf, size_t m_cap) {
  const size_t nb = (m_cap + kPlanChunk - 1) / kPlanChunk + 1;
  uint8_t *b = static_cast<uint8_t *>(buf);
  Scratch r;
  r.item_start = reinterpret_cast<uint64_t *>(b);
  r.block_sum = reinterpret_cast<uint64_t *>(b + 8 * (m_cap + 1));
  r.next = reinterpret_cast<unsigned long long *>(b + 8 * (m_cap + 1) + 8 * nb);
  r.status = reinterpret_cast<int *>(b + 8 * (m_cap + 1) + 8 * nb + 8);
  return r;
}

static int is_capturing(cudaStream_t s, bool *cap) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  *cap = st != cudaStreamCaptureStatusNone;
  return POSPOP_OK;
}

// Workspace of `stream` with room for m arrays (grown if needed).  Caller
// holds ctx.mu.  A call made while the stream is being captured into a
// caller's CUDA graph marks the workspace as captured: the graph keeps its
// addresses, so once the workspace has to grow the old buffer is retired
// (kept until pospopcnt_shutdown) instead of freed.  Graphs made by
// pospopcnt_batch_graph_create have a workspace of their own.
static int get_ws(DevCtx &ctx, cudaStream_t stream, size_t m, Workspace **out) {
  Workspace &w = ctx.ws[stream];
  bool cap = false;
  int rc = is_capturing(stream, &cap);
  if (rc != POSPOP_OK) return rc;
  if (w.buf && w.m_cap >= m) {
    w.captured = w.captured || cap;
    *out = &w;
    return POSPOP_OK;
  }
  if (cap) return POSPOP_ENOMEM;   // no allocation inside a capture: call pospopcnt_reserve first
  size_t cap_m = w.m_cap ? w.m_cap : 65536;
  while (cap_m < m) cap_m *= 2;
  void *buf = nullptr;
  if (cudaMalloc(&buf, scratch_bytes(cap_m)) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ENOMEM;
  }
  if (w.buf) {
    if (w.captured) {
      ctx.retired.push_back(w.buf);   // a caller's graph may replay into it
    } else {
      // the old buffer may still be in use by work queued on this stream
      if (cudaStreamSynchronize(stream) != cudaSuccess) { cudaGetLastError(); }
      cudaFree(w.buf);
    }
  }
  w.buf = buf;
  w.m_cap = cap_m;
  w.scr = scratch_layout(buf, cap_m);
  w.captured = false;
  if (cudaMemsetAsync(w.scr.status, 0, sizeof(int), stream) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  *out = &w;
  return POSPOP_OK;
}

// The three planning kernels; items_fn is plan_items_kernel for the
// array source (CSR offsets or gathered regions).
static int launch_plan(const void *items_fn, const PlanParams &pp, cudaStream_t stream, bool pdl) {
  PlanParams P = pp;
  void *args[] = {&P};
  if (launch_kernel(items_fn, dim3(P.nblocks), dim3(kPlanThreads), args, stream, pdl) !=
          cudaSuccess ||
      launch_kernel(plan_scan_fn(), dim3(1), dim3(kPlanThreads), args, stream, pdl) !=
          cudaSuccess ||
      launch_kernel(plan_apply_fn(), dim3(P.nblocks), dim3(kPlanThreads), args, stream, pdl) !=
          cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(3);
  return POSPOP_OK;
}

int launch_batch_with(DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                      const void *base, const uint64_t *offsets, size_t m, cudaStream_t stream) {
  Scratch scr;
  {
    std::lock_guard<std::mutex> g(ctx.mu);
    Workspace *ws = nullptr;
    const int rc = get_ws(ctx, stream, m, &ws);
    if (rc != POSPOP_OK) return rc;
    scr = ws->scr;
  }
  return launch_batch_scratch(ctx, t, w, counts, base, offsets, m, scr, stream);
}

int launch_batch_scratch(const DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                         const void *base, const uint64_t *offsets, size_t m,
                         const Scratch &scr, cudaStream_t stream) {
  if (cudaMemsetAsync(scr.status, 0, sizeof(int), stream) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  const BatchTune &bt = t.batch[width_group(w)];
  PlanParams pp;
  pp.gptrs = nullptr;
  pp.glens = nullptr;
  pp.offsets = offsets;
  pp.m = m;
  pp.base_addr = (uint64_t)base;
  pp.item_start = scr.item_start;
  pp.block_sum = scr.block_sum;
  pp.next = scr.next;
  pp.status = scr.status;
  memcpy(pp.item_rows, bt.item_rows, sizeof pp.item_rows);
  pp.nblocks = (uint32_t)((m + kPlanChunk - 1) / kPlanChunk);
  int rc = launch_plan(plan_items_fn(), pp, stream, t.pdl != 0);
  if (rc != POSPOP_OK) return rc;

  BatchParams bp;
  bp.gptrs = nullptr;
  bp.glens = nullptr;
  bp.base = static_cast<const uint8_t *>(base);
  bp.offsets = offsets;
  bp.m = m;
  bp.counts = counts;
  bp.w = w;
  bp.item_start = scr.item_start;
  bp.next = scr.next;
  bp.status = scr.status;
  memcpy(bp.item_rows, bt.item_rows, sizeof bp.item_rows);
  bp.grab = bt.grab;
  bp.regroup = t.regroup;
  const Variant *vp = &batch_variant(bt.variant);
  if (w == 256) {   // the two-parity kernel with the tuned block shape
    const int pick = pick_shape(batch256_variant_count(), batch256_variant, 1, *vp);
    if (pick < 0) return POSPOP_EINVAL;
    vp = &batch256_variant(pick);
  }
  const Variant &v = *vp;
  int cps = bt.ctas_per_sm < ctx.occ_batch[bt.variant] ? bt.ctas_per_sm
                                                                 : ctx.occ_batch[bt.variant];
  if (cps < 1) cps = 1;
  void *args[] = {&bp};
  if (launch_kernel(v.fn, dim3((unsigned)(ctx.sms * cps)), dim3(v.bs), args, stream,
                    t.pdl != 0) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(1);
  return POSPOP_OK;
}

// ---------------------------------------------------------------------------
// Gathered regions and word-selected counts.
// ---------------------------------------------------------------------------
static int launch_gather_with(DevCtx &ctx, const TuneTable &t, int w, unsigned long long *counts,
                              const uint64_t *ptrs, const uint64_t *lens, size_t n,
                              cudaStream_t stream) {
  Scratch scr;
  {
    std::lock_guard<std::mutex> g(ctx.mu);
    Workspace *ws = nullptr;
    const int rc = get_ws(ctx, stream, n, &ws);
    if (rc != POSPOP_OK) return rc;
    scr = ws->scr;
  }
  if (cudaMemsetAsync(scr.status, 0, sizeof(int), stream) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  const BatchTune &bt = t.batch[width_group(w)];
  PlanParams pp;
  memset(&pp, 0, sizeof pp);
  pp.gptrs = ptrs;
  pp.glens = lens;
  pp.m = n;
  pp.item_start = scr.item_start;
  pp.block_sum = scr.block_sum;
  pp.next = scr.next;
  pp.status = scr.status;
  memcpy(pp.item_rows, bt.item_rows, sizeof pp.item_rows);
  pp.nblocks = (uint32_t)((n + kPlanChunk - 1) / kPlanChunk);
  const int prc = launch_plan(plan_items_gather_fn(), pp, stream, t.pdl != 0);
  if (prc != POSPOP_OK) return prc;
  BatchParams bp;
  memset(&bp, 0, sizeof bp);
  bp.gptrs = ptrs;
  bp.glens = lens;
  bp.m = n;
  bp.counts = counts;
  bp.w = w;
  bp.item_start = scr.item_start;
  bp.next = scr.next;
  bp.status = scr.status;
  memcpy(bp.item_rows, bt.item_rows, sizeof bp.item_rows);
  bp.grab = bt.grab;
  bp.regroup = t.regroup;
  const Variant *vp = &gather_variant(bt.variant);
  if (w == 256) {   // the two-parity kernel with the tuned block shape
    const int pick = pick_shape(gather256_variant_count(), gather256_variant, 1, *vp);
    if (pick < 0) return POSPOP_EINVAL;
    vp = &gather256_variant(pick);
  }
  const Variant &v = *vp;
  int cps = std::min(bt.ctas_per_sm, ctx.occ_batch[bt.variant]);
  if (cps < 1) cps = 1;
  void *bargs[] = {&bp};
  if (launch_kernel(v.fn, dim3((unsigned)(ctx.sms * cps)), dim3(v.bs), bargs, stream,
                    t.pdl != 0) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(1);
  return POSPOP_OK;
}

static int launch_select_with(DevCtx &ctx, const TuneTable &t, int w,
                              unsigned long long *counts, const void *words, size_t n,
                              const void *select, cudaStream_t stream) {
  const uint64_t W = (uint64_t)w / 8;
  const uint64_t nbytes = n * W;
  const uint64_t p0 = (uint64_t)words, e = p0 + nbytes;
  SelectParams Q;
  StreamParams &P = Q.sp;
  const uint64_t A = p0 & ~15ull;
  P.s.A = reinterpret_cast<const uint8_t *>(A);
  P.s.head = (uint32_t)(p0 - A);
  P.s.G = (((e + 15u) & ~15ull) - A) >> 4;
  P.s.tail = (uint32_t)(e - (A + 16u * (P.s.G - 1)));
  P.counts = counts;
  P.w = w;
  P.rot = (8u * P.s.head) & (uint32_t)(w - 1);
  P.regroup = 0;
  Q.bits = static_cast<const uint8_t *>(select);
  Q.nbits = n;
  Q.nbytes = 4 * ((n + 31) / 32);
  Q.wlog = w == 8 ? 0u : w == 16 ? 1u : w == 32 ? 2u : 3u;
  Q.chunk0 = 0;
  Q.nstaged = 0;
  Q.sel_bytes = 0;
  Q.sel_base = nullptr;
  Q.sel_bit0 = 0;
  Q.status = nullptr;
  Q.wait_cycles = t.wait_cycles;
  const uint64_t R = (P.s.G + 31) >> 5;
  // Staged form: enough chunks wholly inside the span (16 rows; not chunk 0
  // when the span or the bitmap starts inside a 16-byte block, not the
  // partial last granule, and none whose bitmap bytes, rounded out to
  // 16-byte blocks, pass the end of the readable bitmap) to give every warp
  // of the grid at least two.  A chunk from 1 on never reads bitmap bytes
  // before the bitmap's start (its bits start at least 512 * CNT - h >= 128
  // bits in).
  {
    const int si = t.staged ? 4 * ((int)t.staged - 1) + (int)Q.wlog : 0;
    const Variant &sv = select_staged_variant(si);
    const uint64_t warps = (uint64_t)ctx.sms * (uint64_t)(sv.bs / 32);
    const uint64_t CNT = 16u >> Q.wlog;
    const int64_t h = (int64_t)(P.s.head >> Q.wlog);
    const uint64_t mb = (uintptr_t)select & 15u;       // bitmap bytes past a 16-byte block
    const int64_t bit0 = (int64_t)(8 * mb) - h;
    const uint64_t chunk0 = (P.s.head || mb) ? 1 : 0;
    const uint32_t sel_bytes = (uint32_t)(64 * CNT + ((bit0 & 127) ? 16 : 0));
    const uint64_t readable_end = mb + Q.nbytes;       // from the 16-byte-aligned base
    uint64_t chunks = (P.s.G - (P.s.tail < 16 ? 1 : 0)) / 512;
    while (chunks > chunk0 &&
           ((uint64_t)((int64_t)((chunks - 1) * 512 * CNT) + bit0) >> 7) * 16 + sel_bytes >
               readable_end)
      chunks--;
    if (t.staged && ctx.occ_select_staged[si] >= 1 && chunks >= chunk0 + 2 * warps &&
        chunks / warps < (uint64_t(1) << 22)) {   // u32 lane counters: 512 per chunk
      int *status = nullptr;
      {
        std::lock_guard<std::mutex> g(ctx.mu);
        Workspace *ws = nullptr;
        const int rc = get_ws(ctx, stream, 0, &ws);
        if (rc != POSPOP_OK) return rc;
        status = ws->scr.status;
      }
      if (cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess) {
        cudaGetLastError();
        return POSPOP_ECUDA;
      }
      Q.chunk0 = chunk0;
      Q.nstaged = chunks;
      Q.sel_bytes = sel_bytes;
      Q.sel_base = static_cast<const uint8_t *>(select) - mb;
      Q.sel_bit0 = bit0;
      Q.status = status;
      Q.wait_cycles = t.wait_cycles;
      P.row_begin = 0;
      P.row_end = R;
      void *args[] = {&Q};
      if (launch_kernel(sv.fn, dim3(ctx.sms), dim3(sv.bs), args, stream, t.pdl != 0,
                        (size_t)sv.smem) != cudaSuccess) {
        cudaGetLastError();
        return POSPOP_ECUDA;
      }
      note_launches(1);
      return POSPOP_OK;
    }
  }
  // the selection kernel is ALU-heavier than the plain count and runs best
  // in a single wave (measured on GB300): cap the blocks per SM at occupancy
  TuneTable ts = t;
  StreamTune &st = ts.stream[width_group(w)][size_class(R)];
  if (st.ctas_per_sm > ctx.occ_stream[st.variant]) st.ctas_per_sm = ctx.occ_stream[st.variant];
  const StreamPlan pl = plan_stream(ctx, ts, w, R);
  // the selection kernels come in the tune table's block shapes (flush depth
  // 16), four word sizes each; take the planned block shape
  const int shape = pick_shape(select_variant_count(), select_variant, 4, stream_variant(pl.variant));
  if (shape < 0) return POSPOP_EINVAL;
  const Variant &v = select_variant(shape + (int)Q.wlog);
  for (uint64_t rb = 0; rb < R; rb += pl.rows_per_launch) {
    P.row_begin = rb;
    P.row_end = (R - rb > pl.rows_per_launch) ? rb + pl.rows_per_launch : R;
    void *args[] = {&Q};
    if (launch_kernel(v.fn, dim3(pl.grid), dim3(pl.block), args, stream, t.pdl != 0) !=
        cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    note_launches(1);
  }
  return POSPOP_OK;
}

// ---------------------------------------------------------------------------
// Host-memory path.
// ---------------------------------------------------------------------------
static int ensure_staging(DevCtx &ctx) {
  Staging &st = ctx.st;
  if (st.ready) return POSPOP_OK;
  bool ok = cudaStreamCreateWithFlags(&st.copy, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&st.comp, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&st.dcounts, 256 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMallocHost(&st.hcounts, 256 * sizeof(unsigned long long)) == cudaSuccess;
  for (int b = 0; ok && b < kStageBufs; b++)
    ok = cudaMalloc(&st.buf[b], kStageChunk) == cudaSuccess &&
         cudaEventCreateWithFlags(&st.copied[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&st.consumed[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_staging(st);
    return POSPOP_ENOMEM;
  }
  st.ready = true;
  return POSPOP_OK;
}

static int host_count(DevCtx &ctx, int w, uint64_t *counts, const void *bytes, size_t nbytes) {
  const void *dev_bytes = nullptr;
  const PtrKind kc = classify(counts, ctx.device, nullptr);
  const PtrKind kb = classify(bytes, ctx.device, &dev_bytes);
  if ((kc != kPinned && kc != kPageable) || (kb != kPinned && kb != kPageable)) return POSPOP_EPTR;
  std::lock_guard<std::mutex> g(ctx.host_mu);
  int rc = ensure_staging(ctx);
  if (rc != POSPOP_OK) return rc;
  Staging &st = ctx.st;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g2(ctx.mu);
    t = ctx.tune;
  }
  if (cudaMemsetAsync(st.dcounts, 0, 256 * sizeof(unsigned long long), st.comp) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  const bool staged = kb == kPageable;
  if (!staged) {
    // Pinned memory: the kernel reads it in place over the CPU-GPU link.
    rc = launch_stream_with(ctx, t, w, st.dcounts, dev_bytes, nbytes, st.comp);
    if (rc != POSPOP_OK) return rc;
  } else {
    const uint8_t *src = static_cast<const uint8_t *>(bytes);
    size_t chunk = 0;
    for (size_t off = 0; off < nbytes; off += kStageChunk, chunk++) {
      const int b = (int)(chunk % kStageBufs);
      const size_t len = nbytes - off < kStageChunk ? nbytes - off : kStageChunk;
      // chunk starts are multiples of 64 MiB from the start, so every chunk
      // starts on a word boundary and its counters line up with the whole's
      if (cudaStreamWaitEvent(st.copy, st.consumed[b], 0) != cudaSuccess ||
          cudaMemcpyAsync(st.buf[b], src + off, len, cudaMemcpyHostToDevice, st.copy) !=
              cudaSuccess ||
          cudaEventRecord(st.copied[b], st.copy) != cudaSuccess ||
          cudaStreamWaitEvent(st.comp, st.copied[b], 0) != cudaSuccess) {
        cudaGetLastError();
        return POSPOP_ECUDA;
      }
      rc = launch_stream_with(ctx, t, w, st.dcounts, st.buf[b], len, st.comp);
      if (rc != POSPOP_OK) return rc;
      if (cudaEventRecord(st.consumed[b], st.comp) != cudaSuccess) {
        cudaGetLastError();
        return POSPOP_ECUDA;
      }
    }
  }
  if (cudaMemcpyAsync(st.hcounts, st.dcounts, (size_t)w * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, st.comp) != cudaSuccess ||
      cudaStreamSynchronize(st.comp) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  for (int j = 0; j < w; j++) counts[j] += st.hcounts[j];
  return POSPOP_OK;
}

}  // namespace pospop

using namespace pospop;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *pospopcnt_strerror(int code) {
  switch (code) {
    case POSPOP_OK: return "success";
    case POSPOP_EINVAL: return "invalid argument (NULL pointer with nonzero size, bad width, or decreasing offsets)";
    case POSPOP_EPTR: return "pointer is not addressable by the current device (or of the wrong kind)";
    case POSPOP_ECUDA: return "CUDA runtime error or kernel launch failure";
    case POSPOP_ENOMEM: return "out of device or pinned memory (or allocation needed during graph capture)";
    case POSPOP_ETIMEDOUT: return "timed out";
    case POSPOP_EBUSY: return "busy: no free slot or memory budget";
    case POSPOP_ERANGE: return "size beyond the supported maximum";
    default: return "unknown status code";
  }
}

int pospopcnt_init(int device) {
  int rc = POSPOP_OK;
  DevCtx *c = ctx_for_device(device, &rc);
  if (!c) return rc;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return POSPOP_OK;
}

void pospopcnt_shutdown(void) {
  std::lock_guard<std::mutex> g(g_mu);
  for (int d = 0; d < kMaxDevices; d++) {
    if (g_ctx[d] && g_ctx[d]->ready) {
      std::lock_guard<std::mutex> g1(g_ctx[d]->mu);
      std::lock_guard<std::mutex> g2(g_ctx[d]->host_mu);
      free_ctx(*g_ctx[d]);
    }
  }
}

int pospopcnt_async(int w, uint64_t *counts, const void *bytes, size_t nbytes, void *stream) {
  if (!valid_w_single(w)) return POSPOP_EINVAL;
  if (nbytes == 0) return POSPOP_OK;
  if (!counts || !bytes) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *db = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(bytes, c->device, &db))
    return POSPOP_EPTR;
  return launch_stream(*c, w, (unsigned long long *)const_cast<void *>(dc), db, nbytes,
                       static_cast<cudaStream_t>(stream));
}

static int typed_count(int w, uint64_t *counts, const void *words, size_t n) {
  if (n == 0) return POSPOP_OK;
  if (!counts || !words) return POSPOP_EINVAL;
  const size_t W = (size_t)w / 8;
  if (n > SIZE_MAX / W) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *dw = nullptr;
  const PtrKind kc = classify(counts, c->device, &dc);
  const PtrKind kw = classify(words, c->device, &dw);
  if (kc == kBadPtr || kw == kBadPtr) return POSPOP_EPTR;
  const bool dev_c = kc == kDev, dev_w = kw == kDev;
  if (dev_c != dev_w) return POSPOP_EPTR;
  if (!dev_c) return host_count(*c, w, counts, words, n * W);
  rc = launch_stream(*c, w, (unsigned long long *)const_cast<void *>(dc), dw, n * W, nullptr);
  if (rc != POSPOP_OK) return rc;
  if (cudaStreamSynchronize(nullptr) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return POSPOP_OK;
}

int pospopcnt_u8(uint64_t counts[8], const uint8_t *words, size_t n) {
  return typed_count(8, counts, words, n);
}
int pospopcnt_u16(uint64_t counts[16], const uint16_t *words, size_t n) {
  return typed_count(16, counts, words, n);
}
int pospopcnt_u32(uint64_t counts[32], const uint32_t *words, size_t n) {
  return typed_count(32, counts, words, n);
}
int pospopcnt_u64(uint64_t counts[64], const uint64_t *words, size_t n) {
  return typed_count(64, counts, words, n);
}

int pospopcnt_batch(int w, uint64_t *counts, const void *base, const uint64_t *offsets, size_t m,
                    void *stream) {
  if (!valid_w_multi(w)) return POSPOP_EINVAL;
  if (m == 0) return POSPOP_OK;
  if (!counts || !base || !offsets) return POSPOP_EINVAL;
  if (m > (SIZE_MAX / 8) / 256 - 1) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *db = nullptr, *doff = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(base, c->device, &db) ||
      !device_addressable(offsets, c->device, &doff))
    return POSPOP_EPTR;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  return launch_batch_with(*c, t, w, (unsigned long long *)const_cast<void *>(dc), db,
                           static_cast<const uint64_t *>(doff), m,
                           static_cast<cudaStream_t>(stream));
}

int pospopcnt_gather(int w, uint64_t *counts, const uint64_t *ptrs, const uint64_t *lens,
                     size_t n, void *stream) {
  if (!valid_w_multi(w)) return POSPOP_EINVAL;
  if (n == 0) return POSPOP_OK;
  if (!counts || !ptrs || !lens) return POSPOP_EINVAL;
  if (n > (SIZE_MAX / 8) / 256 - 1) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *dp = nullptr, *dl = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(ptrs, c->device, &dp) ||
      !device_addressable(lens, c->device, &dl))
    return POSPOP_EPTR;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  return launch_gather_with(*c, t, w, (unsigned long long *)const_cast<void *>(dc),
                            static_cast<const uint64_t *>(dp), static_cast<const uint64_t *>(dl), n,
                            static_cast<cudaStream_t>(stream));
}

int pospopcnt_masked(int w, uint64_t *counts, const void *words, size_t n, const void *select,
                     void *stream) {
  if (!(w == 8 || w == 16 || w == 32 || w == 64)) return POSPOP_EINVAL;
  if (n == 0) return POSPOP_OK;
  if (!counts || !words || !select) return POSPOP_EINVAL;
  const size_t W = (size_t)w / 8;
  if (((uintptr_t)words % W) != 0 || ((uintptr_t)select % 4) != 0) return POSPOP_EINVAL;
  if (n > SIZE_MAX / W) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *dw = nullptr, *ds = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(words, c->device, &dw) ||
      !device_addressable(select, c->device, &ds))
    return POSPOP_EPTR;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  return launch_select_with(*c, t, w, (unsigned long long *)const_cast<void *>(dc), dw, n, ds,
                            static_cast<cudaStream_t>(stream));
}

int pospopcnt_multi(size_t n, const int *w, uint64_t *const *counts, const void *const *ptrs,
                    const size_t *nbytes, void *stream) {
  if (n == 0) return POSPOP_OK;
  if (!w || !counts || !ptrs || !nbytes) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  // every count is checked before anything is launched
  std::vector<ServeReq> reqs;
  reqs.reserve(n);
  uint64_t rows = 0;
  for (size_t i = 0; i < n; i++) {
    if (!valid_w(w[i])) return POSPOP_EINVAL;
    if (nbytes[i] == 0) continue;
    if (!counts[i] || !ptrs[i]) return POSPOP_EINVAL;
    const void *dc = nullptr, *dp = nullptr;
    if (!device_addressable(counts[i], c->device, &dc) ||
        !device_addressable(ptrs[i], c->device, &dp))
      return POSPOP_EPTR;
    ServeReq r{};   // item0 0: every item of the count is in this launch
    r.ptr = dp;
    r.nbytes = nbytes[i];
    r.w = w[i];
    r.items = 0;
    r.out = (unsigned long long *)const_cast<void *>(dc);
    reqs.push_back(r);
    rows += serve_rows(dp, nbytes[i]);
  }
  if (reqs.empty()) return POSPOP_OK;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  // the launch shape of the single-array entry for the group's mean count
  // size (w = 32 group: counts mix widths)
  const StreamTune &st = t.stream[width_group(32)][size_class(rows / reqs.size())];
  const Variant &sv = stream_variant(st.variant);
  // Groups of large counts (every warp of the grid would get at least 128
  // rows of the mean count, so its per-count flush, fold and block barriers
  // cost little): the single-array kernel's grid-stride schedule over the
  // group's rows, in the single-array entry's waves, one launch ramp and one
  // tail for the whole group.  (Four 96 MiB counts, 40 rows a warp each, ran
  // in 77.5 us this way against 72.1 us as work items; four 1 GiB counts,
  // 431 rows a warp, at 7355 GB/s against 6.8-6.9 TB/s as work items.)
  {
    const uint64_t nw = (uint64_t)c->sms * (uint64_t)std::max(1, st.ctas_per_sm) *
                        (uint64_t)(sv.bs / 32);
    uint64_t max_rows = 0;
    for (const ServeReq &r : reqs) max_rows = std::max(max_rows, serve_rows(r.ptr, r.nbytes));
    if (rows / reqs.size() >= 128 * nw && max_rows / nw < t.max_rows_per_warp &&
        max_rows < (uint64_t(1) << 32) && nw < (uint64_t(1) << 32)) {
      const Variant &mv = multi_stream_variant(st.variant);
      static thread_local ServeParams Q;   // about 10 KiB: not on the caller's stack
      memset(&Q, 0, offsetof(ServeParams, req));
      for (size_t k0 = 0; k0 < reqs.size(); k0 += kServeMax) {
        const size_t cnt = std::min<size_t>(kServeMax, reqs.size() - k0);
        uint64_t first = 0;   // row 0 of count k in this launch's row sequence
        for (size_t k = 0; k < cnt; k++) {
          Q.req[k] = reqs[k0 + k];
          Q.req[k].items = (uint32_t)(first % nw);   // the kernel's starting phase
          first += serve_rows(Q.req[k].ptr, Q.req[k].nbytes);
        }
        Q.n = (uint32_t)cnt;
        void *args[] = {&Q};
        if (launch_kernel(mv.fn, dim3((unsigned)(nw / (sv.bs / 32))), dim3(mv.bs), args,
                          static_cast<cudaStream_t>(stream), t.pdl != 0) != cudaSuccess) {
          cudaGetLastError();
          return POSPOP_ECUDA;
        }
        note_launches(1);
      }
      return POSPOP_OK;
    }
  }
  // Otherwise work items of at most the `multi` entry's rows and at least
  // 8, wave-aligned over the whole group, so that a group of small counts
  // still spreads over the GPU; contiguous or strided items per the entry.
  int vi = find_variant(true, sv.bs, sv.minb, sv.depth, sv.hint);
  if (vi < 0) vi = t.batch[width_group(32)].variant;
  const Variant &v = multi_variant(vi);
  const uint32_t ir = serve_light_rows(*c, vi, rows, t.multi_rows, 8);
  static thread_local ServeParams P;   // about 10 KiB: not on the caller's stack
  memset(&P, 0, offsetof(ServeParams, req));
  // strided items use 32-bit row arithmetic in the kernel
  uint64_t biggest = 0;
  for (const ServeReq &r : reqs) biggest = std::max(biggest, serve_rows(r.ptr, r.nbytes));
  P.strided = (t.multi_strided && biggest < (uint64_t(1) << 32)) ? 1u : 0u;
  const uint64_t wpb = (uint64_t)v.bs / 32;
  for (size_t k0 = 0; k0 < reqs.size(); k0 += kServeMax) {
    const size_t cnt = std::min<size_t>(kServeMax, reqs.size() - k0);
    uint64_t items = 0;
    for (size_t k = 0; k < cnt; k++) {
      ServeReq r = reqs[k0 + k];
      r.items = (uint32_t)((serve_rows(r.ptr, r.nbytes) + ir - 1) / ir);
      r.rows = ir;
      P.item_start[k] = items;
      P.req[k] = r;
      items += r.items;
    }
    P.item_start[cnt] = items;
    P.n = (uint32_t)cnt;
    P.total = items;
    // a persistent grid of at most one wave: each warp takes items i, i + NW,
    // ... in the kernel's grid-stride loop (four 1 GiB counts in one launch:
    // one item per warp in 28 waves of short-lived blocks read at 6.78 TB/s
    // against 7.13 TB/s for four single launches)
    const uint64_t wave = (uint64_t)c->sms * (uint64_t)c->occ_multi[vi];
    const uint64_t grid = std::min<uint64_t>((items + wpb - 1) / wpb, wave);
    // a launch of few counts takes the small parameter block
    static thread_local ServeParamsSmall S;
    const bool small = cnt <= (size_t)kServeSmall;
    if (small) shrink_params(P, S);
    void *args[] = {small ? static_cast<void *>(&S) : static_cast<void *>(&P)};
    if (launch_kernel(small ? multi_small_variant(vi).fn : v.fn, dim3((unsigned)grid), dim3(v.bs),
                      args, static_cast<cudaStream_t>(stream), t.pdl != 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    note_launches(1);
  }
  return POSPOP_OK;
}

int pospopcnt_batch_status(void *stream) {
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  int *status = nullptr;
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->ws.find(s);
    if (it == c->ws.end() || !it->second.buf) return POSPOP_OK;
    status = it->second.scr.status;
  }
  int h = 0;
  if (cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return h == 0 ? POSPOP_OK : h == POSPOP_ETIMEDOUT ? POSPOP_ETIMEDOUT : POSPOP_EINVAL;
}

int pospopcnt_reserve(size_t m_max, void *stream) {
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  std::lock_guard<std::mutex> g(c->mu);
  Workspace *ws = nullptr;
  return get_ws(*c, static_cast<cudaStream_t>(stream), m_max ? m_max : 1, &ws);
}

int pospopcnt_host(int w, uint64_t *counts, const void *bytes, size_t nbytes) {
  if (!valid_w_single(w)) return POSPOP_EINVAL;
  if (nbytes == 0) return POSPOP_OK;
  if (!counts || !bytes) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  return host_count(*c, w, counts, bytes, nbytes);
}

int pospopcnt_roofline_read(const void *bytes, size_t nbytes, uint64_t *sum, void *stream) {
  if (nbytes == 0) return POSPOP_OK;
  if (!bytes || !sum) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *db = nullptr, *ds = nullptr;
  if (!device_addressable(bytes, c->device, &db) || !device_addressable(sum, c->device, &ds))
    return POSPOP_EPTR;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RoofTune rt;
  bool pdl;
  long long wait_cycles;
  int *status = nullptr;
  {
    std::lock_guard<std::mutex> g(c->mu);
    rt = c->tune.roof;
    pdl = c->tune.pdl != 0;
    wait_cycles = c->tune.wait_cycles;
    if (roofline_variant(rt.variant).smem > 0) {   // bulk-copy form: the stream's status word
      Workspace *ws = nullptr;
      rc = get_ws(*c, s, 0, &ws);
      if (rc != POSPOP_OK) return rc;
      status = ws->scr.status;
    }
  }
  if (status && cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return launch_roofline_with(*c, rt, db, nbytes, (unsigned long long *)const_cast<void *>(ds),
                              status, wait_cycles, s, pdl);
}

int pospopcnt_plan(int w, size_t nbytes, uint32_t plan[8]) {
  if (!valid_w_single(w) || !plan) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  const uint64_t G = (nbytes + 15) / 16;
  const uint64_t R = (G + 31) / 32;
  const StreamPlan p = plan_stream(*c, t, w, R);
  const Variant &v = stream_variant(p.variant);
  plan[0] = p.grid;
  plan[1] = p.block;
  plan[2] = (uint32_t)v.depth;
  plan[3] = (uint32_t)v.hint;
  plan[4] = (uint32_t)p.cls;
  plan[5] = (uint32_t)(R > 0xffffffffu ? 0xffffffffu : R);
  plan[6] = (uint32_t)p.launches;
  plan[7] = (uint32_t)p.cps;
  return POSPOP_OK;
}

int pospopcnt_tune_check(const char *path, int *bad_line) {
  if (bad_line) *bad_line = 0;
  if (!path) return POSPOP_EINVAL;
  std::string text;
  if (!read_file(path, &text)) return POSPOP_EINVAL;
  TuneTable t;
  int line = 0;
  const int rc = parse_tune(text.c_str(), &t, &line);
  if (bad_line) *bad_line = rc == POSPOP_OK ? 0 : line;
  return rc;
}

int pospopcnt_tune_load(const char *path) {
  if (!path) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  std::string text;
  if (!read_file(path, &text)) return POSPOP_EINVAL;
  TuneTable t;
  rc = parse_tune(text.c_str(), &t);
  if (rc != POSPOP_OK) return rc;
  t.set_source(path);
  std::lock_guard<std::mutex> g(c->mu);
  c->tune = t;
  return POSPOP_OK;
}

int pospopcnt_tune_describe(char *buf, size_t len) {
  if (!buf || len == 0) return POSPOP_EINVAL;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  std::string s;
  {
    std::lock_guard<std::mutex> g(c->mu);
    s = format_tune(*c, c->tune);
  }
  snprintf(buf, len, "%s", s.c_str());
  return s.size() < len ? POSPOP_OK : POSPOP_ERANGE;
}

// A graph made by pospopcnt_batch_graph_create owns the scratch it was
// captured with (allocated before the capture, freed by
// pospopcnt_graph_destroy), so no later call of the library (a larger batch
// on the same stream, pospopcnt_shutdown) can free memory the graph replays
// into.  `done` is recorded after every replay: destroy waits for it before
// freeing the scratch, and the status query waits for it before reading.
struct pospop_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  Scratch scr;
  int device = -1;
};

static void free_graph(pospop_graph *h) {
  if (h->done) cudaEventSynchronize(h->done);   // the last replay has finished
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->done) cudaEventDestroy(h->done);
  if (h->ws) cudaFree(h->ws);
  cudaGetLastError();
  delete h;
}

int pospopcnt_batch_graph_create(int w, uint64_t *counts, const void *base,
                                 const uint64_t *offsets, size_t m, void *stream, void **graph) {
  if (!graph || !stream) return POSPOP_EINVAL;   // the legacy stream cannot be captured
  *graph = nullptr;
  if (!valid_w_multi(w) || m == 0 || !counts || !base || !offsets) return POSPOP_EINVAL;
  if (m > (SIZE_MAX / 8) / 256 - 1) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  const void *dc = nullptr, *db = nullptr, *doff = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(base, c->device, &db) ||
      !device_addressable(offsets, c->device, &doff))
    return POSPOP_EPTR;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool cap = false;
  rc = is_capturing(s, &cap);
  if (rc != POSPOP_OK) return rc;
  if (cap) return POSPOP_EINVAL;   // the graph is captured on `stream` itself
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  pospop_graph *h = new pospop_graph();
  h->device = c->device;
  h->ws_bytes = scratch_bytes(m);
  if (cudaMalloc(&h->ws, h->ws_bytes) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_graph(h);
    return POSPOP_ENOMEM;
  }
  h->scr = scratch_layout(h->ws, m);
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    free_graph(h);
    return POSPOP_ECUDA;
  }
  rc = launch_batch_scratch(*c, t, w, (unsigned long long *)const_cast<void *>(dc), db,
                            static_cast<const uint64_t *>(doff), m, h->scr, s);
  const cudaError_t e = cudaStreamEndCapture(s, &h->graph);
  if (rc == POSPOP_OK && e != cudaSuccess) rc = POSPOP_ECUDA;
  if (rc == POSPOP_OK && cudaGraphInstantiate(&h->exec, h->graph, 0) != cudaSuccess)
    rc = POSPOP_ECUDA;
  // the status word starts clear (the graph clears it again on every replay)
  if (rc == POSPOP_OK && (cudaMemset(h->scr.status, 0, sizeof(int)) != cudaSuccess ||
                          cudaEventRecord(h->done, s) != cudaSuccess))
    rc = POSPOP_ECUDA;
  if (rc != POSPOP_OK) {
    cudaGetLastError();
    free_graph(h);
    return rc;
  }
  *graph = h;
  return POSPOP_OK;
}

int pospopcnt_graph_launch(void *graph, void *stream) {
  if (!graph) return POSPOP_EINVAL;
  pospop_graph *h = static_cast<pospop_graph *>(graph);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaGraphLaunch(h->exec, s) != cudaSuccess || cudaEventRecord(h->done, s) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(4);
  return POSPOP_OK;
}

int pospopcnt_graph_status(void *graph) {
  if (!graph) return POSPOP_EINVAL;
  pospop_graph *h = static_cast<pospop_graph *>(graph);
  int prev = -1;
  cudaGetDevice(&prev);
  int host = 0;
  const bool ok = cudaSetDevice(h->device) == cudaSuccess &&
                  cudaEventSynchronize(h->done) == cudaSuccess &&
                  cudaMemcpy(&host, h->scr.status, sizeof(int), cudaMemcpyDeviceToHost) ==
                      cudaSuccess &&
                  cudaMemset(h->scr.status, 0, sizeof(int)) == cudaSuccess;
  if (prev >= 0) cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return host == 0 ? POSPOP_OK : POSPOP_EINVAL;
}

int pospopcnt_graph_workspace(void *graph, void **addr, size_t *bytes) {
  if (!graph) return POSPOP_EINVAL;
  const pospop_graph *h = static_cast<const pospop_graph *>(graph);
  if (addr) *addr = h->ws;
  if (bytes) *bytes = h->ws_bytes;
  return POSPOP_OK;
}

int pospopcnt_graph_destroy(void *graph) {
  if (!graph) return POSPOP_EINVAL;
  pospop_graph *h = static_cast<pospop_graph *>(graph);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  free_graph(h);
  if (prev >= 0) cudaSetDevice(prev);
  return POSPOP_OK;
}

uint64_t pospopcnt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"

// pospop_tune.cu -- the autotuner behind pospopcnt_autotune: times every
// launch candidate of the single-array kernel per width group and size
// class, of the batched kernel on a ragged batch per width group, and of the
// roofline read kernel, and
// installs the fastest of each (a candidate must beat the current entry by
// 1%, so measurement noise does not flip near-equal choices).  Timing is with CUDA events on the tuning
// stream; counting kernels do not depend on the data values, so the scratch
// buffer holds a fixed byte pattern.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "pospopcnt.h"
#include "pospop_runtime.h"

namespace pospop {
namespace {

struct Timer {
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  bool ok = false;
  Timer() {
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
  }
  // Mean milliseconds per call of fn (which enqueues on s); < 0 on error.
  double time(const std::function<int()> &fn, double budget_ms = 15.0) {
    if (fn() != POSPOP_OK || cudaStreamSynchronize(s) != cudaSuccess) return -1.0;
    float ms = 0.f;
    if (cudaEventRecord(a, s) != cudaSuccess || fn() != POSPOP_OK ||
        cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
      return -1.0;
    int reps = (int)std::min(200.0, std::max(3.0, budget_ms / std::max(ms, 1e-3f)));
    if (cudaEventRecord(a, s) != cudaSuccess) return -1.0;
    for (int i = 0; i < reps; i++)
      if (fn() != POSPOP_OK) return -1.0;
    if (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
      return -1.0;
    return (double)ms / reps;
  }
};

// xorshift64* for the tuning batch's sizes (tuning input only).
struct Rng {
  uint64_t x;
  uint64_t next() {
    x ^= x >> 12;
    x ^= x << 25;
    x ^= x >> 27;
    return x * 0x2545F4914F6CDD1Dull;
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

}  // namespace
}  // namespace pospop

using namespace pospop;

extern "C" int pospopcnt_autotune(size_t max_bytes, const char *path) {
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  if (max_bytes == 0) max_bytes = size_t(1) << 30;
  if (max_bytes < (size_t(1) << 24)) max_bytes = size_t(1) << 24;

  uint8_t *buf = nullptr;
  unsigned long long *counts = nullptr;
  uint64_t *doff = nullptr;
  if (cudaMalloc(&buf, max_bytes + 64) != cudaSuccess ||
      cudaMalloc(&counts, 20000 * 64 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    return POSPOP_ENOMEM;
  }
  cudaMemset(buf, 0xA5, max_bytes + 64);
  cudaMemset(counts, 0, 20000 * 64 * sizeof(unsigned long long));
  Timer tm;
  if (!tm.ok) {
    cudaGetLastError();
    cudaFree(buf);
    cudaFree(counts);
    return POSPOP_ECUDA;
  }

  TuneTable best;
  {
    std::lock_guard<std::mutex> g(c->mu);
    best = c->tune;
  }
  TuneTable cand = best;

  // --- single-array kernel, per width group and size class ------------------
  const size_t rep_bytes[kClasses] = {size_t(16) << 10, size_t(512) << 10, size_t(16) << 20,
                                      size_t(512) << 20, max_bytes};
  const uint32_t minrows_set[] = {1, 2, 4, 8, 16, 32, 64, 128};
  for (int g = 0; g < kWidthGroups; g++) {
    const int w = kGroupWidth[g];
    for (int cls = 0; cls < kClasses; cls++) {
      const size_t nbytes = std::min(rep_bytes[cls], max_bytes);
      const uint64_t rows = (nbytes / 16 + 31) / 32;
      if (size_class(rows) != cls) {   // scratch too small for this class: inherit
        if (cls > 0) best.stream[g][cls] = best.stream[g][cls - 1];
        continue;
      }
      // the incumbent is timed first; a candidate must beat it by 1% (ties
      // and noise keep the current entry)
      double best_ms =
          tm.time([&] { return launch_stream_with(*c, best, w, counts, buf, nbytes, tm.s); });
      if (best_ms <= 0) best_ms = 1e30;
      for (int v = 0; v < stream_variant_count(); v++) {
        for (int cps = 1; cps <= std::max(4, c->occ_stream[v]); cps++) {
          unsigned last_grid = 0;
          for (uint32_t mr : minrows_set) {
            cand = best;
            cand.stream[g][cls] = StreamTune{v, cps, mr};
            const StreamPlan pl = plan_stream(*c, cand, w, rows);
            if (pl.grid == last_grid) continue;   // same launch as the previous min_rows
            last_grid = pl.grid;
            const double ms = tm.time([&] {
              return launch_stream_with(*c, cand, w, counts, buf, nbytes, tm.s);
            });
            if (ms > 0 && ms < 0.99 * best_ms) {
              best_ms = ms;
              best.stream[g][cls] = cand.stream[g][cls];
            }
          }
        }
      }
    }
  }

  // --- batched kernel on a ragged batch (log-uniform sizes, 1 B .. 4 MiB),
  //     per width group --------------------------------------------------------
  {
    Rng rng{0x9E3779B97F4A7C15ull};
    std::vector<uint64_t> off(1, 0);
    const double lo = 0.0, hi = std::log(4.0 * 1048576.0 + 1.0);
    while (off.size() <= 20000) {
      const uint64_t sz = (uint64_t)std::floor(std::exp(lo + rng.uniform() * (hi - lo)));
      if (off.back() + sz > max_bytes) break;
      off.push_back(off.back() + sz);
    }
    const size_t m = off.size() - 1;
    if (m > 0 && cudaMalloc(&doff, off.size() * sizeof(uint64_t)) == cudaSuccess &&
        cudaMemcpy(doff, off.data(), off.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) ==
            cudaSuccess) {
      const uint32_t item_rows_set[] = {63, 127, 255, 511, 1023, 2047};
      const uint32_t grab_set[] = {1, 2, 4};
      for (int g = 0; g < kWidthGroups; g++) {
        const int w = kGroupWidth[g];
        double best_ms = tm.time(
            [&] { return launch_batch_with(*c, best, w, counts, buf + 3, doff, m, tm.s); });
        if (best_ms <= 0) best_ms = 1e30;
        for (int v = 0; v < batch_variant_count(); v++)
          for (int cps = 1; cps <= std::min(c->occ_batch[v], 4); cps++)
            for (uint32_t ir : item_rows_set)
              for (uint32_t gr : grab_set) {
                cand = best;
                cand.batch[g] = BatchTune{v, cps, ir, gr};
                const double ms = tm.time([&] {
                  return launch_batch_with(*c, cand, w, counts, buf + 3, doff, m, tm.s);
                });
                if (ms > 0 && ms < 0.99 * best_ms) {
                  best_ms = ms;
                  best.batch[g] = cand.batch[g];
                }
              }
      }
    }
    cudaGetLastError();
  }

  // --- roofline read kernel -------------------------------------------------
  // (the bulk-copy form reports an expired staging wait in *dstatus; such a
  // candidate is never chosen)
  int *dstatus = nullptr;
  if (cudaMalloc(&dstatus, sizeof(int)) == cudaSuccess &&
      cudaMemset(dstatus, 0, sizeof(int)) == cudaSuccess) {
    auto status_ok = [&] {
      int h = -1;
      return cudaMemcpy(&h, dstatus, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && h == 0;
    };
    double best_ms = tm.time([&] {
      return launch_roofline_with(*c, best.roof, buf, max_bytes, counts, dstatus,
                                  best.wait_cycles, tm.s, best.pdl != 0);
    });
    if (best_ms <= 0 || !status_ok()) best_ms = 1e30;
    for (int v = 0; v < roofline_variant_count(); v++)
      for (int cps = 1; cps <= 4 * c->occ_roof[v]; cps++) {
        const RoofTune rt{v, cps};
        const double ms = tm.time([&] {
          return launch_roofline_with(*c, rt, buf, max_bytes, counts, dstatus, best.wait_cycles,
                                      tm.s, best.pdl != 0);
        });
        if (!status_ok()) break;
        if (ms > 0 && ms < 0.99 * best_ms) {
          best_ms = ms;
          best.roof = rt;
        }
      }
  }
  if (dstatus) cudaFree(dstatus);

  cudaStreamSynchronize(tm.s);
  if (doff) cudaFree(doff);
  cudaFree(counts);
  cudaFree(buf);
  cudaGetLastError();

  best.set_source("autotuned");
  std::string text;
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->tune = best;
    text = format_tune(*c, best);
  }
  if (path) {
    FILE *f = fopen(path, "wb");
    if (!f) return POSPOP_EINVAL;
    fwrite(text.data(), 1, text.size(), f);
    fclose(f);
  }
  return POSPOP_OK;
}

// pospop_tune.cu -- the autotuner behind pospopcnt_autotune: times every
// launch candidate of the single-array kernel per width group and size
// class; of the batched kernel per width group (launch shape on a mix of a
// ragged and a tiny-array batch, work-item rows per array size class); of
// the serving kernel per serving size class (work-item rows under load and
// at light load); and of the roofline read kernel, and installs the fastest
// of each (a candidate must beat the current entry by 1%, so measurement
// noise does not flip near-equal choices).  Timing is with CUDA events on
// the tuning stream; counting kernels do not depend on the data values, so
// the scratch buffer holds a fixed byte pattern.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
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

// A tuning batch: arrays with sizes log-uniform on [lo, hi] bytes laid back
// to back from the scratch buffer's byte 3 (unaligned starts), at most
// max_arrays of them and max_bytes bytes in all; CSR offsets on the device.
struct TuneBatch {
  uint64_t *doff = nullptr;
  size_t m = 0;
  ~TuneBatch() {
    if (doff) cudaFree(doff);
  }
  bool make(Rng &rng, double lo, double hi, size_t max_arrays, size_t max_bytes) {
    std::vector<uint64_t> off(1, 0);
    const double a = std::log(lo), b = std::log(hi + 1.0);
    while (off.size() <= max_arrays) {
      const uint64_t sz = (uint64_t)std::floor(std::exp(a + rng.uniform() * (b - a)));
      if (off.back() + sz + 3 > max_bytes) break;
      off.push_back(off.back() + sz);
    }
    m = off.size() - 1;
    if (m == 0) return false;
    if (cudaMalloc(&doff, off.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMemcpy(doff, off.data(), off.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }
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
  // Each class is scored on a spread of sizes inside it, each time relative
  // to the incumbent's and summed (a shape that suits the top of a class can
  // cost the bottom of it: one wave against two of the 32 MiB .. 1 GiB class
  // differs by a fifth at 64 MiB and not at all at 1 GiB).  Calls rotate over
  // slices of the scratch buffer, so arrays below the L2 size are still read
  // from DRAM wherever the buffer holds several slices.
  const size_t mix[kClasses][3] = {
      {size_t(16) << 10, 0, 0},
      {size_t(512) << 10, 0, 0},
      {size_t(2) << 20, size_t(8) << 20, size_t(32) << 20},
      {size_t(64) << 20, size_t(256) << 20, size_t(1) << 30},
      {max_bytes, 0, 0}};
  const uint32_t minrows_set[] = {1, 2, 4, 8, 16, 32, 64, 128};
  for (int g = 0; g < kWidthGroups; g++) {
    const int w = kGroupWidth[g];
    for (int cls = 0; cls < kClasses; cls++) {
      std::vector<size_t> sizes;
      for (size_t z : mix[cls])
        if (z > 0 && z <= max_bytes && size_class((z / 16 + 31) / 32) == cls) sizes.push_back(z);
      if (sizes.empty()) {   // scratch too small for this class: inherit
        if (cls > 0) best.stream[g][cls] = best.stream[g][cls - 1];
        continue;
      }
      auto run = [&](const TuneTable &t, size_t nbytes) {
        const size_t slots = std::max<size_t>(1, std::min<size_t>(16, max_bytes / nbytes));
        size_t k = 0;
        return tm.time([&] {
          const size_t off = (k++ % slots) * nbytes;
          return launch_stream_with(*c, t, w, counts, buf + off, nbytes, tm.s);
        });
      };
      // the incumbent is timed first; a candidate must beat it by 1% in the
      // summed relative time (ties and noise keep the current entry)
      std::vector<double> base_ms;
      bool ok = true;
      for (size_t z : sizes) {
        const double ms = run(best, z);
        ok = ok && ms > 0;
        base_ms.push_back(ms);
      }
      if (!ok) continue;
      double best_score = (double)sizes.size();
      for (int v = 0; v < stream_variant_count(); v++) {
        for (int cps = 1; cps <= std::max(4, c->occ_stream[v]); cps++) {
          unsigned last_grid = 0;
          for (uint32_t mr : minrows_set) {
            cand = best;
            cand.stream[g][cls] = StreamTune{v, cps, mr};
            // skip a min_rows that gives the class's smallest size the same
            // grid as the previous one (the larger sizes then mostly share
            // the grid cap as well)
            const StreamPlan pl = plan_stream(*c, cand, w, (sizes[0] / 16 + 31) / 32);
            if (pl.grid == last_grid) continue;
            last_grid = pl.grid;
            double score = 0;
            bool good = true;
            for (size_t i = 0; good && i < sizes.size(); i++) {
              const double ms = run(cand, sizes[i]);
              good = ms > 0;
              score += ms / base_ms[i];
            }
            if (good && score < 0.99 * best_score) {
              best_score = score;
              best.stream[g][cls] = cand.stream[g][cls];
            }
          }
        }
      }
    }
  }

  // --- batched kernel, per width group --------------------------------------
  // Launch shape, blocks per SM and grab size are scored on a mix, not on one
  // size: the ragged batch (1 B .. 4 MiB, the workload's shape) and a batch
  // of tiny arrays (1 B .. 1536 B), each timed relative to the incumbent and
  // summed.  Then the work-item rows of each array size class, each on a
  // batch of arrays of that class only.
  {
    Rng rng{0x9E3779B97F4A7C15ull};
    TuneBatch ragged, tiny, cls[kBatchClasses];
    const double cls_lo[kBatchClasses] = {1, 2049, 32769, 1048577};
    const double cls_hi[kBatchClasses] = {2048, 32768, 1048576, 16777216};
    bool ok = ragged.make(rng, 1, 4.0 * 1048576, 20000, max_bytes) &&
              tiny.make(rng, 1, 1536, 20000, max_bytes);
    for (int k = 0; k < kBatchClasses; k++)
      ok = ok && cls[k].make(rng, cls_lo[k], cls_hi[k], 20000, max_bytes);
    // candidate rows per class: up to one item per array for the small classes
    const std::vector<uint32_t> rows_set[kBatchClasses] = {
        {1, 2, 3, 4}, {2, 4, 8, 16, 32, 64}, {16, 32, 63, 127, 255, 511, 1023, 2048},
        {63, 127, 255, 511, 1023, 2047, 4095}};
    const uint32_t grab_set[] = {1, 2, 4};
    for (int g = 0; ok && g < kWidthGroups; g++) {
      const int w = kGroupWidth[g];
      auto run = [&](const TuneTable &t, const TuneBatch &b) {
        return tm.time(
            [&] { return launch_batch_with(*c, t, w, counts, buf + 3, b.doff, b.m, tm.s); });
      };
      const double r0 = run(best, ragged), t0 = run(best, tiny);
      if (r0 <= 0 || t0 <= 0) continue;
      double best_score = 2.0;   // the incumbent: 1 + 1
      for (int v = 0; v < batch_variant_count(); v++)
        for (int cps = 1; cps <= std::min(c->occ_batch[v], 4); cps++)
          for (uint32_t gr : grab_set) {
            cand = best;
            cand.batch[g].variant = v;
            cand.batch[g].ctas_per_sm = cps;
            cand.batch[g].grab = gr;
            const double r = run(cand, ragged), t = run(cand, tiny);
            if (r <= 0 || t <= 0) continue;
            const double score = r / r0 + t / t0;
            if (score < 0.99 * best_score) {
              best_score = score;
              best.batch[g] = cand.batch[g];
            }
          }
      for (int k = 0; k < kBatchClasses; k++) {
        double best_ms = run(best, cls[k]);
        if (best_ms <= 0) best_ms = 1e30;
        for (uint32_t ir : rows_set[k]) {
          cand = best;
          cand.batch[g].item_rows[k] = ir;
          const double ms = run(cand, cls[k]);
          if (ms > 0 && ms < 0.99 * best_ms) {
            best_ms = ms;
            best.batch[g].item_rows[k] = ir;
          }
        }
      }
    }
    cudaGetLastError();
  }

  // --- serving kernel, per serving size class ---------------------------------
  // `rows` (under load): the time of one launch over 64 requests of the class
  // (sizes log-uniform over the class, widths 8 .. 64), per candidate;
  // `light_rows` (light load): the time of one request of the class's middle
  // size (the geometric mean of its bounds) with wave-aligned items of at
  // most the candidate.  The candidates stop at 511 rows: under load, longer
  // items for the large classes lengthened the tail latency of the 0.9-load
  // trace on GB300 although they read a little faster.
  {
    Rng rng{0xD1B54A32D192ED03ull};
    const double lo[kServeClasses] = {64, 1048576, 16777216, 134217728};
    const double hi[kServeClasses] = {1048576, 16777216, 134217728, 268435456};
    const std::vector<uint32_t> rows_set[kServeClasses] = {
        {31, 63, 127}, {63, 127, 255}, {127, 255, 511}, {127, 255, 511}};
    const uint32_t light_set[] = {8, 16, 32, 63, 127, 0};   // 0: the class's `rows`
    const int sv = best.serve_shape;   // the server's launch shape
    std::unique_ptr<ServeParams> P(new ServeParams());
    unsigned long long *dres = nullptr;
    unsigned int *ddone = nullptr, *dflags = nullptr;
    bool ok = cudaMalloc(&dres, 64 * kServeMax * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&ddone, kServeMax * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&dflags, kServeMax * sizeof(unsigned int)) == cudaSuccess &&
              cudaMemset(ddone, 0, kServeMax * sizeof(unsigned int)) == cudaSuccess &&
              cudaMemset(counts, 0, 64 * kServeMax * sizeof(unsigned long long)) == cudaSuccess;
    // one launch over reqs with items of ir rows (counters left clean by the kernel)
    auto launch = [&](const std::vector<ServeReq> &reqs, uint32_t ir) {
      P->n = (uint32_t)reqs.size();
      P->counts = counts;
      P->done = ddone;
      P->host_res = dres;
      P->flags = dflags;
      P->strided = best.serve_strided;
      uint64_t items = 0;
      for (size_t k = 0; k < reqs.size(); k++) {
        const uint64_t it = (serve_rows(reqs[k].ptr, reqs[k].nbytes) + ir - 1) / ir;
        P->item_start[k] = items;
        P->req[k] = reqs[k];
        P->req[k].items = (uint32_t)it;
        P->req[k].item0 = 0;
        P->req[k].slot = (uint32_t)k;
        P->req[k].seq = 1;
        P->req[k].rows = ir;
        items += it;
      }
      P->item_start[reqs.size()] = items;
      P->total = items;
      return serve_launch(sv, *P, tm.s);
    };
    for (int k = 0; ok && k < kServeClasses; k++) {
      // requests of the class, at random places in the scratch buffer
      std::vector<ServeReq> many;
      uint64_t total = 0;
      while (many.size() < 64) {
        const uint64_t nb =
            (uint64_t)std::exp(std::log(lo[k]) + rng.uniform() * (std::log(hi[k]) - std::log(lo[k])));
        if (nb + 64 > max_bytes || total + nb > max_bytes) break;
        const uint64_t at = 3 + (rng.next() % (max_bytes - nb - 3));
        many.push_back(ServeReq{buf + at, nb, (int32_t)(8 << (many.size() % 4)), 0});
        total += nb;
      }
      if (many.empty()) continue;
      double best_ms = tm.time([&] { return launch(many, best.serve[k].rows); });
      if (best_ms <= 0) best_ms = 1e30;
      for (uint32_t ir : rows_set[k]) {
        const double ms = tm.time([&] { return launch(many, ir); });
        if (ms > 0 && ms < 0.99 * best_ms) {
          best_ms = ms;
          best.serve[k].rows = ir;
        }
      }
      const uint64_t mid = std::min<uint64_t>((uint64_t)std::sqrt(lo[k] * hi[k]), max_bytes - 64);
      const std::vector<ServeReq> one = {ServeReq{buf + 3, mid, 16, 0}};
      const uint64_t rows = serve_rows(buf + 3, mid);
      auto light_ir = [&](uint32_t most) {
        return serve_light_rows(*c, sv, rows, std::min(most ? most : best.serve[k].rows,
                                                       best.serve[k].rows));
      };
      best_ms = tm.time([&] { return launch(one, light_ir(best.serve[k].light_rows)); });
      if (best_ms <= 0) best_ms = 1e30;
      for (uint32_t most : light_set) {
        const double ms = tm.time([&] { return launch(one, light_ir(most)); });
        if (ms > 0 && ms < 0.99 * best_ms) {
          best_ms = ms;
          best.serve[k].light_rows = most;
        }
      }
    }
    cudaStreamSynchronize(tm.s);
    if (dres) cudaFree(dres);
    if (ddone) cudaFree(ddone);
    if (dflags) cudaFree(dflags);
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

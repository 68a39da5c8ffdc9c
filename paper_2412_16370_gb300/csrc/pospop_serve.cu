// pospop_serve.cu -- continuous-batching serving loop for pospopcnt
// requests (declared in include/pospopcnt.h, pospop_server_*).
//
// Requests name device-resident input (any pointer, length and w).  A
// request is ADMITTED when the input bytes of all admitted, unfinished
// requests plus its own fit the server's device-memory budget and a slot is
// free.  The tune entry serve_mode picks how admitted requests reach the
// device: by size class (0, described here), or smallest remaining first in
// launches (1), in launches per size class (2) or through a device-side
// queue into one resident grid (3); serve_loop_srf and serve_loop_resident
// below describe those.  Under the size classes, admitted requests that are
// not yet on the GPU are gathered into one batch as soon as one of the
// server's batch streams is free, so requests
// that arrive while others run are counted in the next batch, overlapping on
// the device with the batches already in flight.  Requests fall into size
// classes (below 1 MiB, 16 MiB, 128 MiB, and above), each served by its own
// batch streams with a stream priority that falls as the class grows, and
// the counting grids are not persistent (one work item per warp, so blocks
// retire every few microseconds): whenever a block of a large request's
// batch retires, the block scheduler hands the SM to pending blocks of a
// smaller class first.  This approximates shortest-remaining-first at the
// granularity of work items, which keeps small requests' latency low under
// load without starving large ones (a class is FIFO within itself).  A batch
// is one launch of serve_kernel (pospop_desc.cu) per kServeMax requests: the requests and
// their work-item prefix sums, planned on the host (it knows every
// request's address and length), travel in the kernel's parameter block, so
// a batch is a launch and an event and nothing else.  Each request slot's
// counters and completion counter live in device memory and are left clean
// by the kernel; the warp that finishes a request publishes its counts to
// mapped pinned memory and raises its flag, which the loop polls.  All
// waits are bounded.
//
// Host input.  A server made by pospop_server_create_pooled owns a device
// staging pool of mem_budget bytes, allocated once.  Requests submitted with
// pospop_server_submit_host name host memory: such a request is admitted
// only when a contiguous range of the pool (first fit, 256-byte granules)
// is free for it, so the budget bounds memory that is really allocated; an
// uploader thread copies each admitted request into its range
// (cudaMemcpyAsync on the server's copy stream, then an event that the
// request's batch stream waits for) and hands it to the loop.  The range is
// released when the request completes, that is, after the kernel has read
// it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "pospopcnt.h"
#include "pospop_runtime.h"

namespace pospop {
namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t id;
  int w;
  const void *dptr;            // device address of the input (the pool range for host input)
  size_t nbytes;
  uint64_t *result;
  pospop_completion rec;
  const void *host = nullptr;  // host input, copied into the pool before counting
  uint64_t pool_off = 0;
  uint64_t pool_len = 0;       // 0: no pool range held
  cudaEvent_t ev = nullptr;    // the upload's completion (waited for by the batch stream)
  // dispatch by remaining bytes (serve_mode 1)
  uint32_t gslot = UINT32_MAX; // server-wide request slot
  uint32_t ir = 0;             // rows per work item (fixed at admission)
  uint32_t items_total = 0;    // work items of ir rows
  uint32_t items_next = 0;     // the first item not yet dispatched
  int launches = 0;            // unfinished launches that hold some of its items
  bool flagged = false;        // the device has published its counts
  bool finished = false;       // completed; freed once no launch holds it
};

constexpr uint64_t kPoolGranule = 256;

struct Batch {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  unsigned long long *dcounts = nullptr;  // 64 per request slot, zero between uses
  unsigned int *ddone = nullptr;        // completion counter per request slot, zero between uses
  unsigned long long *hres = nullptr;   // mapped pinned: per-request counts from the device
  unsigned int *hflags = nullptr;       // mapped pinned: per-request done flags
  unsigned long long *dres = nullptr;   // device addresses of the two above
  unsigned int *dflags = nullptr;
  unsigned int seq = 0;
  std::vector<Request *> reqs;          // null once completed
  bool busy = false;
  int level = 0;                        // size class served by this batch's stream
};

// Size classes: request bytes below kClassBound[k] (and not below the bound
// before) go to class k; the last class takes the rest.  Each class has a
// `serve` entry in the tune table (work-item rows at light load and
// otherwise, batch streams running at once, requests per batch).
constexpr size_t kClassBound[kServeClasses - 1] = {size_t(1) << 20, size_t(16) << 20,
                                                   size_t(128) << 20};
constexpr size_t kBatchCap = 1024;      // requests per batch, at most (4 launches of kServeMax)
constexpr uint64_t kMaxServeGrid = uint64_t(1) << 20;
constexpr uint32_t kMinItemRows = 8;    // the shortest light-load work item
constexpr size_t kGlobalSlots = 16384;  // serve_mode 1: request slots, at most
constexpr uint32_t kResRing = 1u << 14;  // serve_mode 3: runs in the queue's rings
constexpr uint32_t kResIndex = 1u << 20; // serve_mode 3: 64-ticket blocks indexed

// The tune-table entries the loop works with (copied once per loop pass).
struct LoopTune {
  int shape;   // the serving kernel's launch shape (tune entry serve_shape)
  ServeTune cls[kServeClasses];
  uint64_t light;
  uint32_t strided;
  uint32_t order;
  int64_t promote_ns;
};

int request_class(size_t nbytes, int levels) {
  int k = 0;
  while (k < kServeClasses - 1 && nbytes >= kClassBound[k]) k++;
  return k < levels ? k : levels - 1;
}

}  // namespace

uint64_t serve_rows(const void *ptr, uint64_t nbytes) {
  if (nbytes == 0) return 0;
  const uint64_t s0 = (uint64_t)ptr, e0 = s0 + nbytes;
  const uint64_t G = (((e0 + 15u) & ~15ull) - (s0 & ~15ull)) >> 4;
  return (G + 31u) >> 5;
}

uint32_t serve_light_rows(const DevCtx &ctx, int variant, uint64_t rows, uint32_t most,
                          uint32_t least_rows) {
  const uint64_t m = most ? most : 1;
  const uint64_t least = least_rows ? std::min<uint64_t>(least_rows, m)
                                    : std::max<uint64_t>(std::min<uint64_t>(kMinItemRows, m), m / 2);
  const Variant &v = serve_variant(variant);
  const uint64_t warps =
      (uint64_t)ctx.sms * (uint64_t)ctx.occ_serve[variant] * (uint64_t)(v.bs / 32);
  const uint64_t waves = (rows + warps * m - 1) / (warps * m);   // >= 1 (rows > 0)
  const uint64_t want = waves ? (rows + waves * warps - 1) / (waves * warps) : m;
  return (uint32_t)std::min(m, std::max(least, want));
}

int serve_launch(int shape, const ServeParams &P, cudaStream_t stream) {
  // one work item per warp: blocks retire as their items finish, so a
  // smaller class's pending blocks can take the SM (the grid-stride loop in
  // the kernel covers any cap)
  const Variant &v = serve_variant(shape);
  const uint64_t wpb = (uint64_t)v.bs / 32;
  uint64_t grid = (P.total + wpb - 1) / wpb;
  if (grid > kMaxServeGrid) grid = kMaxServeGrid;
  if (grid == 0) return POSPOP_OK;
  // a launch of few requests takes the small parameter block
  static thread_local ServeParamsSmall S;
  const bool small = P.n <= (uint32_t)kServeSmall;
  if (small) shrink_params(P, S);
  void *args[] = {small ? static_cast<void *>(&S) : const_cast<ServeParams *>(&P)};
  const void *fn = small ? serve_small_variant(shape).fn : v.fn;
  if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(v.bs), args, 0, stream) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(1);
  return POSPOP_OK;
}

}  // namespace pospop

struct pospop_server {
  pospop::DevCtx *ctx = nullptr;
  size_t budget = 0;
  int max_inflight = 0;
  int levels = 1;                           // size classes in use (by stream priorities)
  std::vector<pospop::Batch> batches;

  std::mutex mu;
  std::condition_variable cv_loop, cv_done;
  std::deque<pospop::Request *> pending;    // submitted, waiting for admission
  std::deque<pospop::Request *> admitted;   // admitted, not yet on the GPU
  std::deque<pospop_completion> finished;   // completions not yet polled
  size_t inflight_bytes = 0;
  int inflight = 0;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0;
  bool stop = false;
  int loop_error = POSPOP_OK;
  std::thread loop;

  // device staging pool for host input (pospop_server_create_pooled)
  uint8_t *pool = nullptr;
  uint64_t pool_bytes = 0, pool_used = 0, pool_hwm = 0;
  std::map<uint64_t, uint64_t> pool_free;      // offset -> length of the free ranges
  std::deque<pospop::Request *> uploads;       // admitted host input, copy not yet enqueued
  int uploading = 0;                           // taken by the uploader, not yet admitted
  std::vector<cudaEvent_t> spare_events;
  cudaStream_t up_stream = nullptr;
  std::condition_variable cv_up;
  bool stop_uploads = false;
  std::thread uploader;

  // serve_mode 1 (read at creation): admitted requests are dispatched by
  // remaining bytes in launches of at most srf_bytes, srf_launches at once,
  // items of srf_rows rows; each request holds a server-wide slot
  int mode = 0;
  uint64_t srf_bytes = 0;
  int srf_launches = 0;
  uint32_t srf_rows = 0;
  unsigned long long *g_dcounts = nullptr;   // 64 per slot (device, zero between uses)
  unsigned int *g_ddone = nullptr;           // completion counter per slot (device)
  unsigned long long *g_hres = nullptr, *g_dres = nullptr;   // mapped pinned results
  unsigned int *g_hflags = nullptr, *g_dflags = nullptr;     // mapped pinned flags
  std::vector<uint32_t> g_free;              // free slots

  // serve_mode 3: the resident grid and its queue (see pospop_resident.cu)
  pospop::ResRun *r_hruns = nullptr, *r_hruns_dev = nullptr;   // mapped host ring
  pospop::ResCtl *r_hctl = nullptr, *r_hctl_dev = nullptr;     // mapped control block
  pospop::ResRun *r_druns = nullptr;                           // device ring
  uint32_t *r_idx = nullptr;
  pospop::ResState *r_st = nullptr;
  cudaStream_t r_stream = nullptr;
  cudaEvent_t r_done = nullptr;
  int r_variant = 0;
  unsigned r_grid = 0;
};

namespace pospop {
namespace {

void free_batch(Batch &b) {
  if (b.hres) cudaFreeHost(b.hres);
  if (b.hflags) cudaFreeHost(b.hflags);
  if (b.dcounts) cudaFree(b.dcounts);
  if (b.ddone) cudaFree(b.ddone);
  if (b.done) cudaEventDestroy(b.done);
  if (b.s) cudaStreamDestroy(b.s);
  b = Batch();
  cudaGetLastError();
}

uint64_t request_rows(const Request *r) { return serve_rows(r->dptr, r->nbytes); }

// Work-item rows of a batch of `rows` rows of class `level`.  Under load
// the class's `rows`.  While the server is lightly loaded, shorter items
// spread a request over more warps, so its latency is a few short items:
// at most the class's light_rows L (0: `rows`) and at least half of that,
// chosen so that the number of items is a whole multiple of the GPU's
// resident warps where the batch is large enough (every SM takes part and
// there is no partial last wave).  Much shorter items than that cost more
// than they gain: each warp then runs more item set-ups and final
// accumulations for the same bytes (measured on GB300 for a lone 128 MiB
// request: 54-row items in two waves took 35.4 us against 29.8 us for
// 127-row items in one).
uint32_t batch_item_rows(const pospop_server &srv, const LoopTune &lt, int level, uint64_t rows,
                         size_t load_bytes) {
  const ServeTune &st = lt.cls[level];
  if (load_bytes >= lt.light) return st.rows;
  return serve_light_rows(*srv.ctx, lt.shape, rows,
                          std::min(st.light_rows ? st.light_rows : st.rows, st.rows));
}

// Enqueue one batch of the requests in b.reqs on b.s (loop thread only):
// one launch per kServeMax requests, then the batch event.  Requests are
// ordered smallest first, so that small requests' work items come first.
int launch_batch(pospop_server &srv, Batch &b, const LoopTune &lt, size_t load_bytes) {
  std::stable_sort(b.reqs.begin(), b.reqs.end(),
                   [](const Request *x, const Request *y) { return x->nbytes < y->nbytes; });
  const int n = (int)b.reqs.size();
  b.seq = b.seq + 1 == 0 ? 1 : b.seq + 1;
  uint64_t rows = 0;
  for (const Request *r : b.reqs) rows += request_rows(r);
  // item rows of the requests' class (a promoted batch runs on a smaller
  // class's stream); all requests of a batch are of one class
  const int cls = b.reqs.empty() ? b.level : request_class(b.reqs[0]->nbytes, srv.levels);
  const uint32_t ir = batch_item_rows(srv, lt, cls, rows, load_bytes);
  // host input: the batch stream waits for the requests' copies into the pool
  for (const Request *r : b.reqs)
    if (r->ev && cudaStreamWaitEvent(b.s, r->ev, 0) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
  static thread_local ServeParams P;   // about 8 KiB: not on the loop thread's stack
  for (int k0 = 0; k0 < n; k0 += kServeMax) {
    const int cnt = std::min(kServeMax, n - k0);
    P.n = (uint32_t)cnt;
    P.counts = b.dcounts;
    P.done = b.ddone;
    P.host_res = b.dres;
    P.flags = b.dflags;
    P.strided = lt.strided;   // requests are at most the budget: far below 2^32 rows
    uint64_t items = 0;
    for (int k = 0; k < cnt; k++) {
      const Request *r = b.reqs[k0 + k];
      const uint64_t it = (request_rows(r) + ir - 1) / ir;
      P.item_start[k] = items;
      P.req[k] = ServeReq{r->dptr, (uint64_t)r->nbytes, r->w, (uint32_t)it, nullptr,
                          0u, (uint32_t)(k0 + k), b.seq, ir};
      items += it;
      if (it == 0) {   // nothing to count: done as soon as the loop looks
        memset(b.hres + 64 * (size_t)(k0 + k), 0, 64 * sizeof(unsigned long long));
        __atomic_store_n(b.hflags + k0 + k, b.seq, __ATOMIC_RELEASE);
      } else {
        // the slot may still hold this sequence number from 2^32 batches
        // ago: only the kernel may raise it now (seq is never 0)
        __atomic_store_n(b.hflags + k0 + k, 0u, __ATOMIC_RELAXED);
      }
    }
    P.item_start[cnt] = items;
    P.total = items;
    if (items == 0) continue;
    const int rc = serve_launch(lt.shape, P, b.s);
    if (rc != POSPOP_OK) return rc;
  }
  if (cudaEventRecord(b.done, b.s) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  return POSPOP_OK;
}

// First fit of `len` bytes (a multiple of kPoolGranule) in the pool's free
// ranges; caller holds srv.mu.
bool pool_take(pospop_server &srv, uint64_t len, uint64_t *off) {
  for (auto it = srv.pool_free.begin(); it != srv.pool_free.end(); ++it) {
    if (it->second < len) continue;
    *off = it->first;
    const uint64_t rest = it->second - len, at = it->first + len;
    srv.pool_free.erase(it);
    if (rest) srv.pool_free.emplace(at, rest);
    srv.pool_used += len;
    srv.pool_hwm = std::max(srv.pool_hwm, srv.pool_used);
    return true;
  }
  return false;
}

// Return a range to the pool, merged with free neighbours; caller holds srv.mu.
void pool_give(pospop_server &srv, uint64_t off, uint64_t len) {
  srv.pool_used -= len;
  auto next = srv.pool_free.lower_bound(off);
  if (next != srv.pool_free.end() && off + len == next->first) {
    len += next->second;
    next = srv.pool_free.erase(next);
  }
  if (next != srv.pool_free.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      prev->second += len;
      return;
    }
  }
  srv.pool_free.emplace(off, len);
}

// Bookkeeping of a finished request; caller holds srv.mu.  The request is
// freed here unless a launch still holds it (serve_mode 1: a request's
// counts can be published while the launch that counted its last item is
// still counting others); the loop frees it when that launch ends.
void complete(pospop_server &srv, Request *r, int status, int64_t t) {
  if (r->pool_len) pool_give(srv, r->pool_off, r->pool_len);
  if (r->gslot != UINT32_MAX) srv.g_free.push_back(r->gslot);
  if (r->ev) srv.spare_events.push_back(r->ev);
  r->rec.status = status;
  r->rec.t_done_ns = t;
  srv.inflight -= 1;
  srv.inflight_bytes -= r->nbytes;
  srv.completed += 1;
  srv.finished.push_back(r->rec);
  r->finished = true;
  if (r->launches == 0) delete r;
}

// serve_mode 1: a launch that held r has ended (loop thread only).
void drop_launch(Request *r) {
  if (--r->launches == 0 && r->finished) delete r;
}

// serve_mode 1 queue order: the rows a request has not yet had dispatched.
uint64_t rows_left(const Request *r) {
  return (uint64_t)(r->items_total - r->items_next) * r->ir;
}

// Admission by device memory and slots, FIFO (caller holds srv.mu):
// requests leave `pending` while their bytes fit the budget and a slot is
// free (with serve_mode 1 also a server-wide request slot); host input also
// needs a free range of the staging pool and goes to the uploader, the rest
// to `admitted`.  Returns whether any request was admitted.
bool admit(pospop_server &srv, int64_t tnow) {
  bool any = false, to_uploader = false;
  while (!srv.pending.empty() && srv.inflight < srv.max_inflight &&
         srv.inflight_bytes + srv.pending.front()->nbytes <= srv.budget) {
    Request *r = srv.pending.front();
    if (srv.mode >= 1 && srv.g_free.empty()) break;   // wait for a request slot
    if (r->host && r->nbytes > 0) {
      const uint64_t len = (r->nbytes + kPoolGranule - 1) / kPoolGranule * kPoolGranule;
      uint64_t off = 0;
      if (!pool_take(srv, len, &off)) break;   // wait for pool space
      r->pool_off = off;
      r->pool_len = len;
      r->dptr = srv.pool + off;
      if (!srv.spare_events.empty()) {
        r->ev = srv.spare_events.back();
        srv.spare_events.pop_back();
      }
    }
    srv.pending.pop_front();
    if (srv.mode >= 1) {
      r->gslot = srv.g_free.back();
      srv.g_free.pop_back();
    }
    r->rec.t_admit_ns = tnow;
    srv.inflight += 1;
    srv.inflight_bytes += r->nbytes;
    if (r->host) {
      srv.uploads.push_back(r);
      srv.uploading += 1;
      to_uploader = true;
    } else {
      srv.admitted.push_back(r);
    }
    any = true;
  }
  if (to_uploader) srv.cv_up.notify_one();
  return any;
}

// The loop thread owns the batches and every request it has taken out of
// the admitted queue; the mutex guards only the queues and counters, and no
// CUDA call is made while holding it.
void serve_loop(pospop_server *srv) {
  cudaSetDevice(srv->ctx->device);
  std::vector<Batch *> finished_batches;
  std::vector<Request *> done_reqs;
  uint32_t iter = 0;
  int64_t last_activity = now_ns();
  std::vector<std::pair<Batch *, std::vector<Request *>>> to_launch;
  LoopTune lt{};
  while (true) {
    bool progress = false;
    {
      std::lock_guard<std::mutex> g(srv->ctx->mu);
      lt.shape = srv->ctx->tune.serve_shape;
      for (int k = 0; k < kServeClasses; k++) lt.cls[k] = srv->ctx->tune.serve[k];
      lt.light = srv->ctx->tune.serve_light;
      lt.strided = srv->ctx->tune.serve_strided;
      lt.order = srv->ctx->tune.serve_order;
      lt.promote_ns = (int64_t)srv->ctx->tune.serve_promote_us * 1000;
    }
    // 1. completions, without the lock: requests whose flag the device has
    //    raised, and whole batches whose event has fired (which frees the
    //    batch's stream and request slots; a request still unflagged then
    //    failed on the device)
    finished_batches.clear();
    done_reqs.clear();
    const bool sweep = (++iter & 255u) == 0;   // periodic event check (device failures)
    for (Batch &b : srv->batches) {
      if (!b.busy) continue;
      size_t open = 0;
      for (size_t k = 0; k < b.reqs.size(); k++) {
        Request *r = b.reqs[k];
        if (!r) continue;
        if (__atomic_load_n(b.hflags + k, __ATOMIC_ACQUIRE) != b.seq) {
          open++;
          continue;
        }
        if (r->result)
          for (int j = 0; j < r->w; j++) r->result[j] = b.hres[64 * k + j];
        r->rec.status = POSPOP_OK;
        done_reqs.push_back(r);
        b.reqs[k] = nullptr;
      }
      // the event frees the stream and slots; ask only when every request is
      // flagged (or on the periodic sweep, to catch a failed launch)
      if (open > 0 && !sweep) continue;
      const cudaError_t q = cudaEventQuery(b.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) cudaGetLastError();
      for (size_t k = 0; k < b.reqs.size(); k++) {
        Request *r = b.reqs[k];
        if (!r) continue;
        if (q == cudaSuccess && __atomic_load_n(b.hflags + k, __ATOMIC_ACQUIRE) == b.seq) {
          if (r->result)
            for (int j = 0; j < r->w; j++) r->result[j] = b.hres[64 * k + j];
          r->rec.status = POSPOP_OK;
        } else {
          r->rec.status = POSPOP_ECUDA;
        }
        done_reqs.push_back(r);
        b.reqs[k] = nullptr;
      }
      finished_batches.push_back(&b);
    }
    to_launch.clear();
    bool stop_now = false;
    size_t load_bytes = 0;   // device bytes in flight, as the launches saw them
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      const int64_t tnow = now_ns();
      for (Request *r : done_reqs) complete(*srv, r, r->rec.status, tnow);
      for (Batch *b : finished_batches) {
        b->reqs.clear();
        b->busy = false;
      }
      if (!done_reqs.empty() || !finished_batches.empty()) {
        progress = true;
        srv->cv_done.notify_all();
      }
      // 2. admission by device memory and slots (FIFO)
      if (admit(*srv, tnow)) progress = true;
      // 3. admitted requests go, by size class and in admission order, into
      //    the next free batch of their class (while fewer than the class's
      //    `streams` batches are running; at most `cap` requests a batch)
      if (!srv->admitted.empty()) {
        Batch *free_b[kServeClasses] = {nullptr, nullptr, nullptr, nullptr};
        uint32_t running[kServeClasses] = {0, 0, 0, 0};
        for (Batch &b : srv->batches) {
          if (b.busy)
            running[b.level]++;
          else if (!free_b[b.level])
            free_b[b.level] = &b;
        }
        for (int k = 0; k < kServeClasses; k++)
          if (running[k] >= lt.cls[k].streams) free_b[k] = nullptr;
        std::vector<Request *> take[kServeClasses];
        std::deque<Request *> keep;
        for (Request *r : srv->admitted) {
          const int k = request_class(r->nbytes, srv->levels);
          if (free_b[k])
            take[k].push_back(r);   // candidates, trimmed to the class's cap below
          else
            keep.push_back(r);
        }
        for (int k = 0; k < kServeClasses; k++) {
          const size_t cap = std::min<size_t>(kBatchCap, lt.cls[k].cap);
          if (take[k].size() <= cap) continue;
          // serve_order 1: the smallest requests of the class first
          // (shortest-remaining-first among the waiting), else admission order
          if (lt.order)
            std::stable_sort(take[k].begin(), take[k].end(), [](const Request *x,
                                                                 const Request *y) {
              return x->nbytes < y->nbytes;
            });
          for (size_t j = cap; j < take[k].size(); j++) keep.push_back(take[k][j]);
          take[k].resize(cap);
        }
        // serve_promote: a class whose oldest waiting request has waited
        // longer than the limit may use a free stream of the next smaller
        // class (a higher stream priority) that this pass leaves unused
        Batch *up_b[kServeClasses] = {nullptr, nullptr, nullptr, nullptr};
        std::vector<Request *> up[kServeClasses];
        if (lt.promote_ns > 0) {
          for (int k = kServeClasses - 1; k >= 1; k--) {
            if (!free_b[k - 1] || !take[k - 1].empty() || up_b[k - 1]) continue;
            const size_t cap = std::min<size_t>(kBatchCap, lt.cls[k].cap);
            std::deque<Request *> rest;
            for (Request *r : keep) {
              if (up[k].size() < cap && request_class(r->nbytes, srv->levels) == k &&
                  tnow - r->rec.t_submit_ns > lt.promote_ns)
                up[k].push_back(r);
              else
                rest.push_back(r);
            }
            if (!up[k].empty()) {
              up_b[k - 1] = free_b[k - 1];
              keep.swap(rest);
            }
          }
        }
        srv->admitted.swap(keep);
        for (int k = 0; k < kServeClasses; k++) {
          if (take[k].empty()) continue;
          free_b[k]->busy = true;
          to_launch.emplace_back(free_b[k], std::move(take[k]));
          progress = true;
        }
        for (int k = 1; k < kServeClasses; k++) {
          if (up[k].empty()) continue;
          up_b[k - 1]->busy = true;
          to_launch.emplace_back(up_b[k - 1], std::move(up[k]));
          progress = true;
        }
      }
      load_bytes = srv->inflight_bytes;
      const bool busy = std::any_of(srv->batches.begin(), srv->batches.end(),
                                    [](const Batch &b) { return b.busy; });
      if (srv->stop && !busy && srv->admitted.empty() && srv->pending.empty() &&
          srv->uploading == 0)
        stop_now = true;
      // idle: keep polling for a short while (a new request is picked up
      // within a microsecond), then block on the condition variable
      if (progress || busy) last_activity = tnow;
      if (!progress && !busy && !stop_now && tnow - last_activity > 200000)
        srv->cv_loop.wait_for(lk, std::chrono::milliseconds(50));
    }
    // launches, without the lock
    for (auto &bl : to_launch) {
      Batch &b = *bl.first;
      b.reqs = std::move(bl.second);
      const int64_t tl = now_ns();
      for (Request *r : b.reqs) r->rec.t_launch_ns = tl;
      const int rc = launch_batch(*srv, b, lt, load_bytes);
      if (rc != POSPOP_OK) {
        // nothing of this batch reached the device in a usable state:
        // fail its requests (wait for what was enqueued before reusing it)
        cudaStreamSynchronize(b.s);
        cudaGetLastError();
        std::lock_guard<std::mutex> g(srv->mu);
        srv->loop_error = rc;
        for (Request *r : b.reqs)
          if (r) complete(*srv, r, rc, now_ns());
        b.reqs.clear();
        b.busy = false;
        srv->cv_done.notify_all();
      }
    }
    if (stop_now) break;
    if (!progress) std::this_thread::yield();
  }
}

// serve_mode 1: dispatch by remaining bytes.  Admitted requests wait in
// `queue` ordered by the bytes they have not yet had dispatched; whenever
// one of the first srf_launches highest-priority batch streams is free, a
// launch takes work items from the front of the queue (smallest remaining
// first) up to srf_bytes, so a large request is counted over several
// launches while smaller arrivals overtake it at the next launch.
// serve_mode 2 does the same per level: the queue's requests fall into the
// size classes by the bytes they have left (a contiguous run of the queue
// each), a launch takes requests of one level only and runs on one of that
// level's first srf_launches streams, whose priority falls as the level
// grows, so blocks of smaller work overtake waiting blocks of larger work
// on the device while more large work stays in flight.  Every
// request holds a server-wide slot for its whole life (its counters and
// completion counter add up across launches); the warp that finishes its
// last item publishes the counts and raises the slot's flag with the
// request's tag.  The loop thread owns `queue`, `active` and the dispatch
// batches; the mutex guards only the server's queues and counters.
void serve_loop_srf(pospop_server *srv) {
  cudaSetDevice(srv->ctx->device);
  std::vector<Request *> queue;     // admitted, items left to dispatch
  std::vector<Request *> active;    // dispatched in part or whole, not yet finished
  std::vector<Request *> done_reqs;
  std::vector<Batch *> disp;        // the dispatch batches (streams), all levels
  std::vector<Batch *> disp_lv[kServeClasses];
  const bool leveled = srv->mode == 2;
  const int nlev = leveled ? srv->levels : 1;
  for (Batch &b : srv->batches)
    if (b.level < nlev && (int)disp_lv[b.level].size() < srv->srf_launches) {
      disp_lv[b.level].push_back(&b);
      disp.push_back(&b);
    }
  // the level of a request in the queue, by the rows it has left
  auto level_of = [&](const Request *r) {
    return leveled ? request_class((size_t)rows_left(r) * 512u, srv->levels) : 0;
  };
  static thread_local ServeParams P;   // about 14 KiB: not on the loop thread's stack
  int64_t last_activity = now_ns();
  while (true) {
    bool progress = false;
    int shape;
    uint32_t strided;
    ServeTune cls[kServeClasses];
    uint32_t load_rows[kServeClasses];
    uint64_t light;
    int64_t age_ns;
    {
      std::lock_guard<std::mutex> g(srv->ctx->mu);
      shape = srv->ctx->tune.serve_shape;
      strided = srv->ctx->tune.serve_strided;
      for (int k = 0; k < kServeClasses; k++) {
        cls[k] = srv->ctx->tune.serve[k];
        load_rows[k] = srv->ctx->tune.srf_class_rows[k];
      }
      light = srv->ctx->tune.serve_light;
      age_ns = (int64_t)srv->ctx->tune.srf_age_us * 1000;
    }
    // 1. finished launches free their streams; flagged requests are done;
    //    a request whose launches all finished unflagged failed on the device
    done_reqs.clear();
    for (Batch *b : disp) {
      if (!b->busy) continue;
      const cudaError_t q = cudaEventQuery(b->done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) cudaGetLastError();
      for (Request *r : b->reqs) drop_launch(r);
      b->reqs.clear();
      b->busy = false;
      progress = true;
    }
    for (size_t k = 0; k < active.size();) {
      Request *r = active[k];
      if (!r->flagged &&
          __atomic_load_n(srv->g_hflags + r->gslot, __ATOMIC_ACQUIRE) == (uint32_t)r->id) {
        if (r->result)
          for (int j = 0; j < r->w; j++) r->result[j] = srv->g_hres[64 * (size_t)r->gslot + j];
        r->flagged = true;
        r->rec.status = POSPOP_OK;
      } else if (!r->flagged && r->launches == 0 && r->items_next == r->items_total) {
        r->rec.status = POSPOP_ECUDA;   // every launch finished, no result
      } else {
        k++;
        continue;
      }
      // (a flagged request's slot is written no more: it completes now,
      // and launches that still hold it free it when they end)
      done_reqs.push_back(r);
      active[k] = active.back();
      active.pop_back();
      progress = true;
    }
    // 2. under the lock: completions, admission, newly admitted requests
    std::vector<Request *> incoming;
    bool stop_now = false;
    size_t load_bytes = 0;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      const int64_t tnow = now_ns();
      for (Request *r : done_reqs) complete(*srv, r, r->rec.status, tnow);
      if (!done_reqs.empty()) srv->cv_done.notify_all();
      if (admit(*srv, tnow)) progress = true;
      load_bytes = srv->inflight_bytes;
      incoming.assign(srv->admitted.begin(), srv->admitted.end());
      srv->admitted.clear();
      const bool busy = !queue.empty() || !active.empty() || !incoming.empty() ||
                        std::any_of(disp.begin(), disp.end(), [](Batch *b) { return b->busy; });
      if (srv->stop && !busy && srv->pending.empty() && srv->uploading == 0) stop_now = true;
      if (progress || busy) last_activity = tnow;
      if (!progress && !busy && !stop_now && tnow - last_activity > 200000)
        srv->cv_loop.wait_for(lk, std::chrono::milliseconds(50));
    }
    // 3. newly admitted requests join the queue (empty ones are done at
    //    once); while the server is lightly loaded a request's items follow
    //    its class's light-load rule, else they have srf_rows rows (with
    //    srf_rows 0, the rows of their class's `serve` entry)
    for (Request *r : incoming) {
      const uint64_t rrows = serve_rows(r->dptr, r->nbytes);
      if (load_bytes < light) {
        const ServeTune &st = cls[request_class(r->nbytes, srv->levels)];
        r->ir = serve_light_rows(*srv->ctx, shape, rrows,
                                 std::min(st.light_rows ? st.light_rows : st.rows, st.rows));
      } else {   // the class's serve_srf_class rows, else srf_rows, else (0) its serve rows
        const int k = request_class(r->nbytes, srv->levels);
        r->ir = load_rows[k]     ? load_rows[k]
                : srv->srf_rows  ? srv->srf_rows
                                 : std::max<uint32_t>(1, cls[k].rows);
      }
      r->items_total = (uint32_t)((rrows + r->ir - 1) / r->ir);
      if (r->items_total == 0) {
        if (r->result)
          for (int j = 0; j < r->w; j++) r->result[j] = 0;
        r->rec.status = POSPOP_OK;
        std::lock_guard<std::mutex> g(srv->mu);
        complete(*srv, r, POSPOP_OK, now_ns());
        srv->cv_done.notify_all();
        continue;
      }
      // the slot's flag may hold this request's tag from 2^32 requests ago:
      // clear it, so that only the kernel can raise it
      __atomic_store_n(srv->g_hflags + r->gslot, ~(uint32_t)r->id, __ATOMIC_RELAXED);
      // the queue stays ordered by rows left (after those with as many)
      const uint64_t key = rows_left(r);
      queue.insert(std::upper_bound(queue.begin(), queue.end(), key,
                                    [](uint64_t k, const Request *x) { return k < rows_left(x); }),
                   r);
      progress = true;
    }
    // 4. dispatch: one launch per free dispatch stream, smallest remaining
    //    first (per level with serve_mode 2)
    for (int lv = 0; lv < nlev; lv++) {
      for (Batch *b : disp_lv[lv]) {
        if (b->busy) continue;
        // the level's run of the queue: [lo, hi)
        size_t lo = 0, hi = queue.size();
        if (leveled) {   // the level grows with the rows left: binary searches
          lo = (size_t)(std::partition_point(queue.begin(), queue.end(),
                                             [&](const Request *x) { return level_of(x) < lv; }) -
                        queue.begin());
          hi = (size_t)(std::partition_point(queue.begin() + (std::ptrdiff_t)lo, queue.end(),
                                             [&](const Request *x) { return level_of(x) <= lv; }) -
                        queue.begin());
        }
        if (lo == hi) break;   // nothing of this level: its other streams too
        // the launch takes a prefix of the run, all of it but the last
        // request wholly; that one has fewer rows left than any request
        // after it and goes back to its place in the queue
        uint64_t budget = srv->srf_bytes;
        uint64_t items = 0;
        uint32_t n = 0;
        // one entry of this launch: up to `cap` bytes of r's next items
        auto take_from = [&](Request *r, uint64_t cap) {
          const uint64_t item_bytes = (uint64_t)r->ir * 512u;
          const uint64_t left = r->items_total - r->items_next;
          const uint64_t take = std::min<uint64_t>(left, std::max<uint64_t>(1, cap / item_bytes));
          P.req[n] = ServeReq{r->dptr, (uint64_t)r->nbytes, r->w, r->items_total, nullptr,
                              r->items_next, r->gslot, (uint32_t)r->id, r->ir};
          P.item_start[n] = items;
          items += take;
          budget -= std::min<uint64_t>(budget, take * item_bytes);
          r->items_next += (uint32_t)take;
          r->launches += 1;
          if (r->items_next == (uint32_t)take) {
            r->rec.t_launch_ns = now_ns();   // its first launch
            active.push_back(r);
          }
          b->reqs.push_back(r);
          if (r->ev && cudaStreamWaitEvent(b->s, r->ev, 0) != cudaSuccess) cudaGetLastError();
          n++;
        };
        // serve_srf_age (serve_mode 1): the longest-waiting request, once it
        // has waited that long, takes up to half the launch first (it leaves
        // its place in the queue and goes back by its rows left)
        if (age_ns > 0 && !leveled && hi - lo > 1) {
          const int64_t tnow = now_ns();
          size_t oldest = hi;
          for (size_t q = lo + 1; q < hi; q++)
            if (tnow - queue[q]->rec.t_submit_ns > age_ns &&
                (oldest == hi || queue[q]->rec.t_submit_ns < queue[oldest]->rec.t_submit_ns))
              oldest = q;
          if (oldest < hi) {
            Request *r = queue[oldest];
            queue.erase(queue.begin() + (std::ptrdiff_t)oldest);
            hi--;
            take_from(r, srv->srf_bytes / 2);
            if (r->items_next < r->items_total)
              queue.insert(std::upper_bound(queue.begin(), queue.end(), rows_left(r),
                                            [](uint64_t k, const Request *x) {
                                              return k < rows_left(x);
                                            }),
                           r);
            hi = queue.size();   // (serve_mode 1: the run is the whole queue)
          }
        }
        size_t taken = 0;
        for (size_t q = lo; q < hi; q++) {
          Request *r = queue[q];
          if (n == (uint32_t)kServeMax || budget == 0) break;
          take_from(r, budget);
          taken++;
          if (r->items_next < r->items_total) break;   // the budget is spent
        }
        // requests with every item dispatched leave the queue
        Request *part = taken > 0 && queue[lo + taken - 1]->items_next <
                                         queue[lo + taken - 1]->items_total
                            ? queue[lo + taken - 1]
                            : nullptr;
        queue.erase(queue.begin() + (std::ptrdiff_t)lo,
                    queue.begin() + (std::ptrdiff_t)(lo + taken));
        if (part)
          queue.insert(std::upper_bound(queue.begin(), queue.end(), rows_left(part),
                                        [](uint64_t k, const Request *x) {
                                          return k < rows_left(x);
                                        }),
                       part);
        P.n = n;
        P.total = items;
        P.counts = srv->g_dcounts;
        P.done = srv->g_ddone;
        P.host_res = srv->g_dres;
        P.flags = srv->g_dflags;
        P.strided = strided;
        P.item_start[n] = items;
        int rc = serve_launch(shape, P, b->s);
        if (rc == POSPOP_OK && cudaEventRecord(b->done, b->s) != cudaSuccess) rc = POSPOP_ECUDA;
        b->busy = true;
        if (rc != POSPOP_OK) {
          // the launch did not reach the device in a usable state: wait for
          // every dispatch stream (nothing may still write a slot), retire the
          // other launches, then the requests this launch held get no more
          // dispatches and, unflagged, fail in the next pass
          cudaGetLastError();
          for (Batch *x : disp) cudaStreamSynchronize(x->s);
          cudaGetLastError();
          for (Batch *x : disp) {
            if (x == b || !x->busy) continue;
            for (Request *r : x->reqs) drop_launch(r);
            x->reqs.clear();
            x->busy = false;
          }
          for (Request *r : b->reqs) {
            if (!r->finished) r->items_next = r->items_total;
            drop_launch(r);
          }
          b->reqs.clear();
          b->busy = false;
          queue.erase(std::remove_if(queue.begin(), queue.end(),
                                     [](const Request *r) {
                                       return r->items_next == r->items_total;
                                     }),
                      queue.end());
          std::lock_guard<std::mutex> g(srv->mu);
          srv->loop_error = rc;
        }
        progress = true;
      }
    }
    if (stop_now) break;
    if (!progress) std::this_thread::yield();
  }
}

// serve_mode 3: smallest remaining first through a device-side queue into
// one resident grid (pospop_resident.cu).  The loop keeps the admitted
// requests ordered by the rows they have left, as serve_mode 1 does, and
// publishes runs of their work items from the front whenever the queue's
// unclaimed work (what the grid has not yet taken, from its `head` that the
// doorbell mirrors to host memory) is below serve_srf's <bytes>; the grid
// claims the items in that order, so an arrival waits behind at most that
// much work.  The grid is launched when work arrives and there is none on
// the device, and is told to leave (by the epoch of its launch) after
// serve_resident's idle time without work.  If it leaves for any other
// reason (its own wait for a run ran out, or a device error), every request
// with published items that has not completed fails, and the queue and the
// slots are reset before the next launch.  A run goes into the host ring
// only at a position the doorbell has already copied out of (the doorbell
// mirrors its copy count), and the unclaimed tickets stay far below what
// the 64-ticket index holds.
void serve_loop_resident(pospop_server *srv) {
  cudaSetDevice(srv->ctx->device);
  std::vector<Request *> queue;     // admitted, items left to publish (rows left ascending)
  std::vector<Request *> staging;   // host input whose copy into the pool has not finished
  std::vector<Request *> active;    // published in part or whole, not yet finished
  std::vector<Request *> done_reqs;
  struct Pub {
    uint64_t t0, t1, item_bytes;    // tickets [t0, t1) of one run
  };
  std::deque<Pub> pubs;             // published runs not yet wholly claimed
  uint64_t pub_bytes = 0;           // their bytes
  uint64_t published = 0, tickets = 0, epoch = 0;
  bool running = false, stopping = false;
  int64_t last_work = now_ns(), last_activity = now_ns();
  auto fits = [](uint64_t k, const Request *x) { return k < rows_left(x); };
  auto reset_queue = [&]() {
    // the grid is gone: nothing reads the rings, the index or the slots
    cudaMemsetAsync(srv->r_st, 0, sizeof(ResState), srv->r_stream);
    cudaMemsetAsync(srv->r_druns, 0, sizeof(ResRun) * kResRing, srv->r_stream);
    cudaMemsetAsync(srv->r_idx, 0, sizeof(uint32_t) * kResIndex, srv->r_stream);
    const size_t slots = std::min<size_t>((size_t)srv->max_inflight, kGlobalSlots);
    cudaMemsetAsync(srv->g_dcounts, 0, 64 * sizeof(unsigned long long) * slots, srv->r_stream);
    cudaMemsetAsync(srv->g_ddone, 0, sizeof(unsigned int) * slots, srv->r_stream);
    cudaStreamSynchronize(srv->r_stream);
    cudaGetLastError();
    __atomic_store_n(&srv->r_hctl->published, 0ull, __ATOMIC_RELEASE);
    __atomic_store_n(&srv->r_hctl->head_seen, 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&srv->r_hctl->copied_seen, 0ull, __ATOMIC_RELAXED);
    published = tickets = 0;
    pubs.clear();
    pub_bytes = 0;
  };
  while (true) {
    bool progress = false;
    int shape;
    ServeTune cls[kServeClasses];
    uint32_t load_rows[kServeClasses];
    uint64_t light;
    int64_t idle_ns, wait_ns;
    {
      std::lock_guard<std::mutex> g(srv->ctx->mu);
      shape = srv->r_variant;
      for (int k = 0; k < kServeClasses; k++) {
        cls[k] = srv->ctx->tune.serve[k];
        load_rows[k] = srv->ctx->tune.srf_class_rows[k];
      }
      light = srv->ctx->tune.serve_light;
      idle_ns = (int64_t)srv->ctx->tune.res_idle_us * 1000;
      wait_ns = (int64_t)srv->ctx->tune.res_wait_us * 1000;
    }
    // 1. flags of finished requests
    done_reqs.clear();
    for (size_t k = 0; k < active.size();) {
      Request *r = active[k];
      if (__atomic_load_n(srv->g_hflags + r->gslot, __ATOMIC_ACQUIRE) == (uint32_t)r->id) {
        if (r->result)
          for (int j = 0; j < r->w; j++) r->result[j] = srv->g_hres[64 * (size_t)r->gslot + j];
        r->rec.status = POSPOP_OK;
        done_reqs.push_back(r);
        active[k] = active.back();
        active.pop_back();
        progress = true;
      } else {
        k++;
      }
    }
    // 2. the grid has left
    if (running) {
      const cudaError_t q = cudaEventQuery(srv->r_done);
      if (q != cudaErrorNotReady) {
        if (q != cudaSuccess) cudaGetLastError();
        int status = POSPOP_OK;
        if (cudaMemcpy(&status, &srv->r_st->status, sizeof(int), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
          cudaGetLastError();
          status = POSPOP_ECUDA;
        }
        const bool clean = stopping && q == cudaSuccess && status == POSPOP_OK;
        running = stopping = false;
        progress = true;
        if (!clean) {
          // flags raised before the grid left still count; the rest fail
          for (size_t k = 0; k < active.size(); k++) {
            Request *r = active[k];
            if (__atomic_load_n(srv->g_hflags + r->gslot, __ATOMIC_ACQUIRE) == (uint32_t)r->id) {
              if (r->result)
                for (int j = 0; j < r->w; j++)
                  r->result[j] = srv->g_hres[64 * (size_t)r->gslot + j];
              r->rec.status = POSPOP_OK;
            } else {
              r->rec.status = q == cudaSuccess && status == POSPOP_ETIMEDOUT ? POSPOP_ETIMEDOUT
                                                                            : POSPOP_ECUDA;
              if (r->items_next < r->items_total)   // still queued for its other items
                queue.erase(std::remove(queue.begin(), queue.end(), r), queue.end());
            }
            done_reqs.push_back(r);
          }
          active.clear();
          reset_queue();
        }
      }
    }
    // 3. under the lock: completions, admission, newly admitted requests
    std::vector<Request *> incoming;
    bool stop_now = false, server_stop = false;
    size_t load_bytes = 0;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      const int64_t tnow = now_ns();
      for (Request *r : done_reqs) complete(*srv, r, r->rec.status, tnow);
      if (!done_reqs.empty()) srv->cv_done.notify_all();
      if (admit(*srv, tnow)) progress = true;
      load_bytes = srv->inflight_bytes;
      incoming.assign(srv->admitted.begin(), srv->admitted.end());
      srv->admitted.clear();
      server_stop = srv->stop;
      const bool work = !queue.empty() || !staging.empty() || !active.empty() ||
                        !incoming.empty() || !srv->pending.empty() || srv->uploading > 0;
      if (work) last_work = tnow;
      if (server_stop && !work && !running) stop_now = true;
      if (progress || work || running) last_activity = tnow;
      if (!progress && !work && !running && !stop_now && tnow - last_activity > 200000)
        srv->cv_loop.wait_for(lk, std::chrono::milliseconds(50));
    }
    // 4. newly admitted requests: item rows, flag cleared, into the queue
    //    (host input once its copy into the pool has finished)
    for (Request *r : incoming) {
      const uint64_t rrows = serve_rows(r->dptr, r->nbytes);
      if (load_bytes < light) {
        const ServeTune &st = cls[request_class(r->nbytes, srv->levels)];
        r->ir = serve_light_rows(*srv->ctx, shape, rrows,
                                 std::min(st.light_rows ? st.light_rows : st.rows, st.rows));
      } else {
        const int k = request_class(r->nbytes, srv->levels);
        r->ir = load_rows[k]     ? load_rows[k]
                : srv->srf_rows  ? srv->srf_rows
                                 : std::max<uint32_t>(1, cls[k].rows);
      }
      r->items_total = (uint32_t)((rrows + r->ir - 1) / r->ir);
      if (r->items_total == 0) {
        if (r->result)
          for (int j = 0; j < r->w; j++) r->result[j] = 0;
        std::lock_guard<std::mutex> g(srv->mu);
        complete(*srv, r, POSPOP_OK, now_ns());
        srv->cv_done.notify_all();
        continue;
      }
      __atomic_store_n(srv->g_hflags + r->gslot, ~(uint32_t)r->id, __ATOMIC_RELAXED);
      staging.push_back(r);
      progress = true;
    }
    for (size_t k = 0; k < staging.size();) {
      Request *r = staging[k];
      if (r->ev) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) {
          k++;
          continue;
        }
        if (q != cudaSuccess) cudaGetLastError();
      }
      queue.insert(std::upper_bound(queue.begin(), queue.end(), rows_left(r), fits), r);
      staging[k] = staging.back();
      staging.pop_back();
    }
    // 5. the grid: launch it when there is work and none is on the device;
    //    publish runs while the unclaimed work is below the target
    if (!queue.empty() && !running && !stopping && active.empty() &&
        tickets > kResTicketLimit - (1ull << 32))
      reset_queue();   // the ticket numbers start again (nothing is on the device)
    if (!queue.empty() && !running && !stopping) {
      ResParams P;
      P.hruns = srv->r_hruns_dev;
      P.ctl = srv->r_hctl_dev;
      P.druns = srv->r_druns;
      P.idx = srv->r_idx;
      P.st = srv->r_st;
      P.counts = srv->g_dcounts;
      P.done = srv->g_ddone;
      P.host_res = srv->g_dres;
      P.flags = srv->g_dflags;
      P.C = kResRing;
      P.B = kResIndex;
      P.epoch = ++epoch;
      P.wait_ns = wait_ns;
      const Variant &v = resident_variant(shape);
      void *args[] = {&P};
      if (cudaLaunchKernel(v.fn, dim3(srv->r_grid), dim3(v.bs), args, 0, srv->r_stream) !=
              cudaSuccess ||
          cudaEventRecord(srv->r_done, srv->r_stream) != cudaSuccess) {
        // no grid: every queued request fails
        cudaGetLastError();
        std::lock_guard<std::mutex> g(srv->mu);
        srv->loop_error = POSPOP_ECUDA;
        for (Request *r : queue) complete(*srv, r, POSPOP_ECUDA, now_ns());
        queue.clear();
        srv->cv_done.notify_all();
      } else {
        note_launches(1);
        running = true;
      }
      progress = true;
    }
    if (running && !stopping && !queue.empty()) {
      const uint64_t head = __atomic_load_n(&srv->r_hctl->head_seen, __ATOMIC_RELAXED);
      while (!pubs.empty() && pubs.front().t1 <= head) {
        pub_bytes -= (pubs.front().t1 - pubs.front().t0) * pubs.front().item_bytes;
        pubs.pop_front();
      }
      uint64_t backlog = pub_bytes;   // less what the grid has taken of the first run
      if (!pubs.empty() && head > pubs.front().t0)
        backlog -= (head - pubs.front().t0) * pubs.front().item_bytes;
      const uint64_t run0 = published;
      const uint64_t copied = __atomic_load_n(&srv->r_hctl->copied_seen, __ATOMIC_RELAXED);
      while (!queue.empty() && backlog < srv->srf_bytes) {
        if (published - copied >= kResRing) break;   // the host ring is full
        if (tickets >= kResTicketLimit) break;        // a reset first (above)
        Request *r = queue.front();
        const uint64_t item_bytes = (uint64_t)r->ir * 512u;
        const uint64_t left = r->items_total - r->items_next;
        uint64_t n = std::min<uint64_t>(
            left, std::max<uint64_t>(1, (srv->srf_bytes - backlog + item_bytes - 1) / item_bytes));
        n = std::min<uint64_t>(n, (1ull << kResNBits) - 1);
        // unclaimed tickets stay within the 64-ticket index, with room to spare
        const uint64_t room = (uint64_t)kResIndex * 32u;
        if (tickets + n > head + room) {
          if (tickets >= head + room) break;
          n = head + room - tickets;
        }
        ResRun &run = srv->r_hruns[published & (kResRing - 1)];
        run.ptr = r->dptr;
        run.nbytes = r->nbytes;
        run.key = 0;
        run.left = 0;
        run.w = r->w;
        run.items = r->items_total;
        run.item0 = r->items_next;
        run.n = (uint32_t)n;
        run.slot = r->gslot;
        run.tag = (uint32_t)r->id;
        run.rows = r->ir;
        if (r->items_next == 0) {
          r->rec.t_launch_ns = now_ns();   // its first run
          active.push_back(r);
        }
        pubs.push_back(Pub{tickets, tickets + n, item_bytes});
        pub_bytes += n * item_bytes;
        backlog += n * item_bytes;
        tickets += n;
        published++;
        r->items_next += (uint32_t)n;
        // wholly published requests leave the queue; a split one has the
        // fewest rows left and stays first
        if (r->items_next == r->items_total) queue.erase(queue.begin());
      }
      if (published != run0) {
        __atomic_store_n(&srv->r_hctl->published, (unsigned long long)published, __ATOMIC_RELEASE);
        progress = true;
      }
    }
    // 6. idle: tell the grid to leave (at once when the server is stopping)
    if (running && !stopping && queue.empty() && staging.empty() && active.empty() &&
        (server_stop || now_ns() - last_work > idle_ns)) {
      __atomic_store_n(&srv->r_hctl->stop, (unsigned long long)epoch, __ATOMIC_RELEASE);
      stopping = true;
      progress = true;
    }
    if (stop_now) break;
    if (!progress) std::this_thread::yield();
  }
}

// The uploader: copies admitted host input into its pool range on the copy
// stream, records the copy's event and hands the request to the loop.  A
// pageable source makes cudaMemcpyAsync wait until the bytes are staged, so
// this runs on its own thread, not on the loop's.
void upload_loop(pospop_server *srv) {
  cudaSetDevice(srv->ctx->device);
  while (true) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_up.wait(lk, [&] { return srv->stop_uploads || !srv->uploads.empty(); });
      if (srv->uploads.empty()) break;   // stopping, nothing left
      r = srv->uploads.front();
      srv->uploads.pop_front();
    }
    int rc = POSPOP_OK;
    if (!r->ev && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
      rc = POSPOP_ECUDA;
    if (rc == POSPOP_OK && r->nbytes > 0 &&
        cudaMemcpyAsync(const_cast<void *>(r->dptr), r->host, r->nbytes, cudaMemcpyHostToDevice,
                        srv->up_stream) != cudaSuccess)
      rc = POSPOP_ECUDA;
    if (rc == POSPOP_OK && cudaEventRecord(r->ev, srv->up_stream) != cudaSuccess)
      rc = POSPOP_ECUDA;
    if (rc != POSPOP_OK) cudaGetLastError();
    {
      std::lock_guard<std::mutex> g(srv->mu);
      srv->uploading -= 1;
      if (rc == POSPOP_OK) {
        srv->admitted.push_back(r);
      } else {
        srv->loop_error = rc;
        complete(*srv, r, rc, now_ns());
        srv->cv_done.notify_all();
      }
    }
    srv->cv_loop.notify_one();
  }
}

// Queue one request.  `t_arrival` is its arrival time (the submit time, or a
// load generator's scheduled arrival, so that latency includes any delay in
// submitting it).
int submit_impl(pospop_server *srv, int w, const void *dptr, size_t nbytes, uint64_t *result,
                uint64_t *id, int64_t t_arrival, const void *host = nullptr) {
  Request *r = new Request();
  r->w = w;
  r->dptr = dptr;
  r->host = host;
  r->nbytes = nbytes;
  r->result = result;
  memset(&r->rec, 0, sizeof r->rec);
  r->rec.w = w;
  r->rec.nbytes = nbytes;
  uint64_t rid;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) {
      delete r;
      return POSPOP_EBUSY;
    }
    rid = srv->next_id++;
    r->id = rid;
    r->rec.id = rid;
    r->rec.t_submit_ns = t_arrival;
    srv->pending.push_back(r);
    srv->submitted += 1;
  }
  srv->cv_loop.notify_one();
  if (id) *id = rid;
  return POSPOP_OK;
}

bool valid_width(int w) {
  return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64;
}

// Device address of a request's input, or POSPOP_EPTR.
int request_ptr(pospop_server *srv, const void *bytes, size_t nbytes, const void **dptr) {
  *dptr = bytes;
  if (nbytes == 0) return POSPOP_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, bytes) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_EPTR;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *dptr = a.devicePointer;
    return POSPOP_OK;
  }
  if ((a.type == cudaMemoryTypeDevice && a.device == srv->ctx->device) ||
      a.type == cudaMemoryTypeManaged)
    return POSPOP_OK;
  return POSPOP_EPTR;
}

// Free what a server holds on the device and the host (its threads have
// stopped, nothing of it is in flight).
void free_server(pospop_server *srv) {
  for (Batch &x : srv->batches) free_batch(x);
  if (srv->r_hruns) cudaFreeHost(srv->r_hruns);
  if (srv->r_hctl) cudaFreeHost(srv->r_hctl);
  if (srv->r_druns) cudaFree(srv->r_druns);
  if (srv->r_idx) cudaFree(srv->r_idx);
  if (srv->r_st) cudaFree(srv->r_st);
  if (srv->r_done) cudaEventDestroy(srv->r_done);
  if (srv->r_stream) cudaStreamDestroy(srv->r_stream);
  if (srv->g_dcounts) cudaFree(srv->g_dcounts);
  if (srv->g_ddone) cudaFree(srv->g_ddone);
  if (srv->g_hres) cudaFreeHost(srv->g_hres);
  if (srv->g_hflags) cudaFreeHost(srv->g_hflags);
  for (cudaEvent_t e : srv->spare_events) cudaEventDestroy(e);
  if (srv->pool) cudaFree(srv->pool);
  if (srv->up_stream) cudaStreamDestroy(srv->up_stream);
  cudaGetLastError();
  delete srv;
}

int create_server(size_t mem_budget, int max_inflight, int max_batches, bool pooled,
                  pospop_server **out) {
  if (!out || mem_budget == 0 || max_inflight < 1 || max_inflight > (1 << 20) || max_batches < 1 ||
      max_batches > 64)
    return POSPOP_EINVAL;
  *out = nullptr;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  pospop_server *srv = new pospop_server();
  srv->ctx = c;
  srv->budget = mem_budget;
  srv->max_inflight = max_inflight;
  // one size class per stream priority level (at most kServeClasses), each
  // with max_batches batch streams; class 0 (the smallest requests) gets the
  // greatest priority
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  srv->levels = std::max(1, std::min(kServeClasses, least - greatest + 1));
  srv->batches.resize((size_t)max_batches * (size_t)srv->levels);
  const size_t slots = std::min((size_t)max_inflight, kBatchCap);
  for (size_t i = 0; i < srv->batches.size(); i++) {
    Batch &b = srv->batches[i];
    b.level = (int)(i / (size_t)max_batches);
    const int prio = greatest + b.level;   // numerically lower = higher priority
    const size_t cbytes = 64 * sizeof(unsigned long long) * slots;
    const size_t fbytes = sizeof(unsigned int) * slots;
    if (cudaStreamCreateWithPriority(&b.s, cudaStreamNonBlocking, prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b.dcounts, cbytes) != cudaSuccess ||
        cudaMalloc(&b.ddone, fbytes) != cudaSuccess ||
        cudaMemset(b.dcounts, 0, cbytes) != cudaSuccess ||
        cudaMemset(b.ddone, 0, fbytes) != cudaSuccess ||
        cudaHostAlloc(&b.hres, cbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(&b.hflags, fbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&b.dres), b.hres, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&b.dflags), b.hflags, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      free_server(srv);
      return POSPOP_ENOMEM;
    }
    memset(b.hflags, 0, fbytes);   // seq starts at 1
  }
  {
    std::lock_guard<std::mutex> g(c->mu);
    srv->mode = c->tune.serve_mode;
    srv->srf_bytes = c->tune.srf_bytes;
    srv->srf_launches = std::max(1, std::min(max_batches, (int)c->tune.srf_launches));
    srv->srf_rows = c->tune.srf_rows;
    srv->r_variant = c->tune.serve_shape;
  }
  if (srv->mode == 3) {
    // the queue's rings, control block and state; the grid fills every SM
    const size_t rbytes = sizeof(ResRun) * kResRing;
    int occ = 0;
    const Variant &v = resident_variant(srv->r_variant);
    if (cudaHostAlloc(&srv->r_hruns, rbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(&srv->r_hctl, sizeof(ResCtl), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&srv->r_hruns_dev), srv->r_hruns, 0) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&srv->r_hctl_dev), srv->r_hctl, 0) !=
            cudaSuccess ||
        cudaMalloc(&srv->r_druns, rbytes) != cudaSuccess ||
        cudaMalloc(&srv->r_idx, sizeof(uint32_t) * kResIndex) != cudaSuccess ||
        cudaMalloc(&srv->r_st, sizeof(ResState)) != cudaSuccess ||
        cudaMemset(srv->r_druns, 0, rbytes) != cudaSuccess ||
        cudaMemset(srv->r_idx, 0, sizeof(uint32_t) * kResIndex) != cudaSuccess ||
        cudaMemset(srv->r_st, 0, sizeof(ResState)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&srv->r_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->r_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, v.bs, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      free_server(srv);
      return POSPOP_ENOMEM;
    }
    memset(srv->r_hruns, 0, rbytes);
    memset(srv->r_hctl, 0, sizeof(ResCtl));
    srv->r_grid = (unsigned)(c->sms * occ);
  }
  if (srv->mode >= 1) {
    // server-wide request slots: a request keeps one for its whole life
    const size_t slots = std::min<size_t>((size_t)max_inflight, kGlobalSlots);
    const size_t cbytes = 64 * sizeof(unsigned long long) * slots;
    const size_t fbytes = sizeof(unsigned int) * slots;
    if (cudaMalloc(&srv->g_dcounts, cbytes) != cudaSuccess ||
        cudaMalloc(&srv->g_ddone, fbytes) != cudaSuccess ||
        cudaMemset(srv->g_dcounts, 0, cbytes) != cudaSuccess ||
        cudaMemset(srv->g_ddone, 0, fbytes) != cudaSuccess ||
        cudaHostAlloc(&srv->g_hres, cbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(&srv->g_hflags, fbytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&srv->g_dres), srv->g_hres, 0) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&srv->g_dflags), srv->g_hflags, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      free_server(srv);
      return POSPOP_ENOMEM;
    }
    memset(srv->g_hflags, 0, fbytes);
    for (size_t k = slots; k > 0; k--) srv->g_free.push_back((uint32_t)(k - 1));
  }
  if (pooled) {
    // the staging pool for host input: allocated once, the whole budget
    if (cudaMalloc(&srv->pool, mem_budget) != cudaSuccess ||
        cudaStreamCreateWithFlags(&srv->up_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      free_server(srv);
      return POSPOP_ENOMEM;
    }
    srv->pool_bytes = mem_budget;
    srv->pool_free.emplace(0, mem_budget / kPoolGranule * kPoolGranule);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {   // the zeroed slots are in place
    cudaGetLastError();
    free_server(srv);
    return POSPOP_ECUDA;
  }
  srv->loop = std::thread(srv->mode == 3 ? serve_loop_resident
                          : srv->mode >= 1 ? serve_loop_srf : serve_loop,
                          srv);
  if (pooled) srv->uploader = std::thread(upload_loop, srv);
  *out = srv;
  return POSPOP_OK;
}

}  // namespace
}  // namespace pospop

using namespace pospop;

extern "C" {

int pospop_server_create(size_t mem_budget, int max_inflight, int max_batches,
                         pospop_server **out) {
  return create_server(mem_budget, max_inflight, max_batches, false, out);
}

int pospop_server_create_pooled(size_t mem_budget, int max_inflight, int max_batches,
                                pospop_server **out) {
  return create_server(mem_budget, max_inflight, max_batches, true, out);
}

int pospop_server_submit_host(pospop_server *srv, int w, const void *bytes, size_t nbytes,
                              uint64_t *result, uint64_t *id) {
  if (!srv || !valid_width(w)) return POSPOP_EINVAL;
  if (!srv->pool) return POSPOP_EINVAL;   // not a pooled server
  if (nbytes > 0 && !bytes) return POSPOP_EINVAL;
  if (nbytes > srv->budget) return POSPOP_ERANGE;
  if (nbytes > 0) {
    // host memory only (pinned or pageable); device input goes through
    // pospop_server_submit
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, bytes) != cudaSuccess) {
      cudaGetLastError();
      return POSPOP_EPTR;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return POSPOP_EPTR;
  }
  static const uint8_t kEmpty = 0;
  return submit_impl(srv, w, nullptr, nbytes, result, id, now_ns(), nbytes ? bytes : &kEmpty);
}

int pospop_server_pool_stats(pospop_server *srv, uint64_t stats[3]) {
  if (!srv || !stats) return POSPOP_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  stats[0] = srv->pool_bytes;
  stats[1] = srv->pool_used;
  stats[2] = srv->pool_hwm;
  return POSPOP_OK;
}

int pospop_server_submit(pospop_server *srv, int w, const void *bytes, size_t nbytes,
                         uint64_t *result, uint64_t *id) {
  if (!srv || !valid_width(w)) return POSPOP_EINVAL;
  if (nbytes > 0 && !bytes) return POSPOP_EINVAL;
  if (nbytes > srv->budget) return POSPOP_ERANGE;
  const void *dptr = nullptr;
  const int rc = request_ptr(srv, bytes, nbytes, &dptr);
  if (rc != POSPOP_OK) return rc;
  return submit_impl(srv, w, dptr, nbytes, result, id, now_ns());
}

int pospop_server_poll(pospop_server *srv, pospop_completion *out, int max, int timeout_ms) {
  if (!srv || !out || max < 1) return POSPOP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (srv->finished.empty() && timeout_ms > 0)
    srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                          [&] { return !srv->finished.empty(); });
  if (srv->finished.empty()) return POSPOP_ETIMEDOUT;
  int n = 0;
  while (n < max && !srv->finished.empty()) {
    out[n++] = srv->finished.front();
    srv->finished.pop_front();
  }
  return n;
}

int pospop_server_drain(pospop_server *srv, int timeout_ms) {
  if (!srv) return POSPOP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return srv->completed == srv->submitted; });
  return ok ? POSPOP_OK : POSPOP_ETIMEDOUT;
}

int pospop_server_stats(pospop_server *srv, uint64_t stats[6]) {
  if (!srv || !stats) return POSPOP_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  stats[0] = srv->submitted;
  stats[1] = srv->completed;
  stats[2] = srv->pending.size();
  stats[3] = (uint64_t)srv->inflight;
  stats[4] = srv->inflight_bytes;
  stats[5] = (uint64_t)(int64_t)srv->loop_error;
  return POSPOP_OK;
}

int pospop_server_run_trace(pospop_server *srv, size_t n, const int64_t *arrival_ns,
                            const int32_t *w, const uint64_t *ptrs, const uint64_t *nbytes,
                            uint64_t *results, pospop_completion *out, int timeout_ms) {
  if (!srv || (n > 0 && (!arrival_ns || !w || !ptrs || !nbytes || !out))) return POSPOP_EINVAL;
  if (n == 0) return POSPOP_OK;
  // validate every request before the clock starts
  std::vector<const void *> dptr(n);
  for (size_t i = 0; i < n; i++) {
    if (!valid_width(w[i]) || (nbytes[i] > 0 && ptrs[i] == 0)) return POSPOP_EINVAL;
    if (nbytes[i] > srv->budget) return POSPOP_ERANGE;
    if (i > 0 && arrival_ns[i] < arrival_ns[i - 1]) return POSPOP_EINVAL;
    const int rc = request_ptr(srv, reinterpret_cast<const void *>(ptrs[i]), nbytes[i], &dptr[i]);
    if (rc != POSPOP_OK) return rc;
  }
  uint64_t first_id = 0;
  const int64_t t0 = now_ns();
  for (size_t i = 0; i < n; i++) {
    const int64_t due = t0 + arrival_ns[i];
    while (now_ns() < due) {
    }
    uint64_t rid = 0;
    const int rc = submit_impl(srv, w[i], dptr[i], nbytes[i], results ? results + 64 * i : nullptr,
                               &rid, due);
    if (rc != POSPOP_OK) return rc;
    if (i == 0) first_id = rid;
  }
  // collect the n completions (ids are consecutive when this is the only submitter)
  size_t got = 0;
  std::vector<pospop_completion> buf(4096);
  const int64_t deadline = now_ns() + (int64_t)timeout_ms * 1000000;
  while (got < n) {
    const int64_t left_ms = (deadline - now_ns()) / 1000000;
    if (left_ms <= 0) return POSPOP_ETIMEDOUT;
    const int k = pospop_server_poll(srv, buf.data(), (int)buf.size(),
                                     (int)std::min<int64_t>(left_ms, 100));
    if (k == POSPOP_ETIMEDOUT) continue;
    if (k < 0) return k;
    for (int j = 0; j < k; j++) {
      const uint64_t idx = buf[j].id - first_id;
      if (idx < n) {
        out[idx] = buf[j];
        got++;
      }
    }
  }
  return POSPOP_OK;
}

int pospop_server_destroy(pospop_server *srv) {
  if (!srv) return POSPOP_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv_loop.notify_all();
  if (srv->loop.joinable()) srv->loop.join();   // every request has finished
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop_uploads = true;
  }
  srv->cv_up.notify_all();
  if (srv->uploader.joinable()) srv->uploader.join();
  for (Batch &b : srv->batches)
    if (b.s) cudaStreamSynchronize(b.s);
  if (srv->up_stream) cudaStreamSynchronize(srv->up_stream);
  free_server(srv);
  return POSPOP_OK;
}

}  // extern "C"

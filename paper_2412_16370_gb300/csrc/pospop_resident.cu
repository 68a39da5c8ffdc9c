// pospop_resident.cu -- serve_mode 3's resident grid: one launch that stays
// on the device while the server has work and is fed through a queue in
// memory instead of one launch per batch.
//
// The host appends runs (a run: consecutive work items of one request) to a
// ring in mapped pinned memory and raises `published`.  Warp 0 of block 0 is
// the doorbell: it copies new runs into a ring in device memory (one run
// per lane, 32 at a time), numbers their work items with consecutive
// tickets (a run's first ticket is the sum of the items before it), records
// for every block of 64 tickets the run that holds its first ticket, and
// releases the ticket count.  A ring position is reused only once the run
// in it has been wholly counted (each worker takes one from the run's
// `left` when it is done with the record), and a run's tickets sit in one
// 8-byte key written after its other fields, so a warp that scans the ring
// sees a run whole or not at all.  Every other warp claims one ticket at a
// time (an atomic on `head`, taken only while a released ticket is left, so
// that idle warps do not run ahead), finds its run from the 64-ticket index
// and at most three warp-wide scans of the ring, and counts that work item with
// the paper's per-thread algorithm (Section 4) into the request's slot, as
// the serving kernel does: the warp that finishes a request's last item
// publishes its counts and raises its flag with the request's tag.
//
// Every wait is bounded.  The doorbell leaves when the host writes this
// launch's epoch to `stop`, or when no run has arrived for `wait_ns`
// (status POSPOP_ETIMEDOUT); either way it sets the device-side stop, and
// the workers leave when they see it, or on their own when no run has
// arrived for twice that long.  A worker that holds a ticket not yet
// released waits for it under the same limits.  The last warp to leave
// sets `head` back to the released ticket count (tickets claimed beyond it
// were never released), so the next launch starts where this one ended.
// The host stops the grid only when every published item has been counted.
#include "pospopcnt.h"
#include "pospop_batch.cuh"

namespace pospop {
namespace {

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// The doorbell: copy published runs, number their tickets, release them.
__device__ void doorbell(const ResParams &P, unsigned lane) {
  ResState *st = P.st;
  unsigned long long copied = *reinterpret_cast<volatile unsigned long long *>(&st->copied);
  unsigned long long tickets = *reinterpret_cast<volatile unsigned long long *>(&st->tickets);
  long long last = timer_ns();
  if (lane == 0) *reinterpret_cast<volatile unsigned long long *>(&st->beat) = (unsigned long long)last;
  unsigned nap = 32;
  while (true) {
    // the host's view of the claimed tickets, for its count of unclaimed work
    if (lane == 0)
      *reinterpret_cast<volatile unsigned long long *>(&P.ctl->head_seen) =
          *reinterpret_cast<volatile unsigned long long *>(&st->head);
    const unsigned long long pub = ld_acquire_sys(&P.ctl->published);   // every lane
    if (pub > copied) {
      const unsigned long long j = copied + lane;
      const bool have = j < pub;
      ResRun run{};
      if (have) run = P.hruns[j & (P.C - 1)];   // ordered after this lane's acquire
      const uint32_t n = have ? run.n : 0u;
      uint32_t incl = n;   // inclusive sum of the runs' items over the lanes
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += v;
      }
      // the ring position's previous run must be wholly counted before it
      // is overwritten (bounded: a warp counts an item in microseconds)
      ResRun *d = P.druns + (j & (P.C - 1));
      bool stuck = false;
      if (have) {
        const long long t_in = timer_ns();
        while (ld_acquire_gpu(&d->left) != 0u) {
          if (timer_ns() - t_in > P.wait_ns) {
            stuck = true;
            break;
          }
          __nanosleep(64);
        }
      }
      if (__any_sync(kFull, stuck)) {
        if (lane == 0) atomicExch(&st->status, POSPOP_ETIMEDOUT);
        break;
      }
      if (have) {
        const unsigned long long t0 = tickets + (incl - n);
        d->ptr = run.ptr;
        d->nbytes = run.nbytes;
        d->w = run.w;
        d->items = run.items;
        d->item0 = run.item0;
        d->n = n;
        d->slot = run.slot;
        d->tag = run.tag;
        d->rows = run.rows;
        d->left = n;
        __threadfence();   // the fields before the key that makes the run visible
        *reinterpret_cast<volatile unsigned long long *>(&d->key) = (t0 << kResNBits) | n;
        // the 64-ticket blocks whose first ticket is in this run
        for (unsigned long long b = (t0 + 63) >> 6; (b << 6) < t0 + n; b++)
          P.idx[b & (P.B - 1)] = (uint32_t)j;
      }
      const uint32_t added = __shfl_sync(kFull, incl, 31);
      copied += (pub - copied < 32ull) ? (pub - copied) : 32ull;
      tickets += added;
      __threadfence();   // this lane's runs and index entries first
      __syncwarp();
      last = timer_ns();
      if (lane == 0) {
        *reinterpret_cast<volatile unsigned long long *>(&st->copied) = copied;
        *reinterpret_cast<volatile unsigned long long *>(&st->beat) = (unsigned long long)last;
        st_release_gpu(&st->tickets, tickets);
        *reinterpret_cast<volatile unsigned long long *>(&P.ctl->copied_seen) = copied;
      }
      nap = 32;
      continue;
    }
    if (ld_acquire_sys(&P.ctl->stop) == P.epoch) break;
    if (timer_ns() - last > P.wait_ns) {
      if (lane == 0) atomicExch(&st->status, POSPOP_ETIMEDOUT);
      break;
    }
    __nanosleep(nap);
    nap = nap < 1024 ? nap * 2 : 1024;
  }
  if (lane == 0) {
    *reinterpret_cast<volatile unsigned long long *>(&P.ctl->head_seen) =
        *reinterpret_cast<volatile unsigned long long *>(&st->head);
    __threadfence();
    atomicExch(&st->stop, 1u);
  }
  __syncwarp();
}

// A worker leaves when the doorbell has set the stop, or when no run has
// arrived for twice the doorbell's limit (the doorbell is gone); `since` is
// the worker's own start, so that a doorbell not yet running does not count.
__device__ __forceinline__ bool must_leave(const ResParams &P, long long since) {
  if (ld_acquire_gpu(&P.st->stop)) return true;
  long long beat = (long long)*reinterpret_cast<volatile unsigned long long *>(&P.st->beat);
  if (beat < since) beat = since;
  return timer_ns() - beat > 2 * P.wait_ns;
}

}  // namespace

template <int BS, int MINB, int DEPTH, int HINT>
__global__ void __launch_bounds__(BS, MINB) resident_kernel(const __grid_constant__ ResParams P) {
  constexpr unsigned WPB = BS / 32;
  const unsigned lane = threadIdx.x & 31u;
  ResState *st = P.st;
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    doorbell(P, lane);
  } else {
    // each warp's start time, kept in shared memory: only the idle paths
    // read it, so the count loop keeps its registers (no block barrier here:
    // block 0's doorbell warp takes no part in the workers' loop)
    __shared__ long long since_s[WPB];
    volatile long long *since = since_s + (threadIdx.x >> 5);
    if (lane == 0) *since = timer_ns();
    __syncwarp();
    const Xpose xk = make_xpose(lane);
    unsigned nap = 32;
    while (true) {
      unsigned long long t = ~0ull;
      if (lane == 0) {
        const unsigned long long h = *reinterpret_cast<volatile unsigned long long *>(&st->head);
        if (h < ld_acquire_gpu(&st->tickets)) t = atomicAdd(&st->head, 1ull);
      }
      t = __shfl_sync(kFull, t, 0);
      if (t == ~0ull) {   // nothing released: wait, bounded
        if (__any_sync(kFull, must_leave(P, *since))) break;
        __nanosleep(nap);
        nap = nap < 8192 ? nap * 2 : 8192;
        continue;
      }
      nap = 32;
      // the ticket may have been claimed past the released count: wait
      // until every lane has seen it released (each lane's own acquire, so
      // that its reads of the run and the index below come after it)
      bool gone = false;
      while (!__all_sync(kFull, t < ld_acquire_gpu(&st->tickets))) {
        if (__any_sync(kFull, must_leave(P, *since))) {
          gone = true;
          break;
        }
        __nanosleep(64);
      }
      if (gone) break;
      // the run holding ticket t: at or after the one holding the block's
      // first ticket, and at most 64 runs start in one block
      uint32_t j = P.idx[(t >> 6) & (P.B - 1)];
      int found = -1;
      for (int round = 0; round < 3 && found < 0; round++, j += 32) {
        // the key holds the run's tickets in one word: a run being written
        // into a position is either wholly seen or not at all
        const unsigned long long key = ld_acquire_gpu(&P.druns[(j + lane) & (P.C - 1)].key);
        const unsigned long long t0 = key >> kResNBits;
        const unsigned long long nn = key & ((1ull << kResNBits) - 1);
        const unsigned hit = __ballot_sync(kFull, t >= t0 && t < t0 + nn);
        if (hit) found = (int)(j & (P.C - 1)) + __ffs(hit) - 1;
      }
      if (found < 0) {   // cannot happen with a consistent ring: the grid leaves
        if (lane == 0) {
          atomicExch(&st->status, POSPOP_EINVAL);
          __threadfence();
          atomicExch(&st->stop, 1u);
        }
        break;
      }
      // the run's fields are read where they are used (after the count
      // loop again from memory), so that they do not hold registers the
      // loop needs
      ResRun *rp = P.druns + ((uint32_t)found & (P.C - 1));
      const uint64_t s0 = (uint64_t)rp->ptr, e0 = s0 + rp->nbytes;
      Span s;
      const uint64_t A = s0 & ~15ull;
      s.A = reinterpret_cast<const uint8_t *>(A);
      s.head = (uint32_t)(s0 - A);
      s.G = (((e0 + 15u) & ~15ull) - A) >> 4;
      s.tail = (uint32_t)(e0 - (A + 16u * (s.G - 1)));
      const uint64_t R = span_rows(s);
      const uint32_t rows = rp->rows;
      const uint64_t kk = (uint64_t)rp->item0 + (t - (rp->key >> kResNBits));   // within its request
      const uint64_t r0 = kk * rows;
      const uint64_t nrows = ((r0 + rows < R) ? r0 + rows : R) - r0;
      uint32_t cnt[4] = {0u, 0u, 0u, 0u};
      count_rows<DEPTH, HINT>(s, r0, 1, nrows, lane, xk, cnt, PlainLoader<HINT>{});
      const int w = rp->w;
      const uint32_t rot = (8u * s.head) & (uint32_t)(w - 1);
      const uint32_t slot = rp->slot;
      unsigned long long *out = P.counts + 64ull * slot;
      fold_counts(cnt, w, rot, lane, [&](uint32_t jj, unsigned long long v) {
        if (v) atomicAdd(out + jj, v);
      });
      // completion of the request, as in the serving kernel
      __threadfence();
      unsigned last = 0;
      if (lane == 0) last = atomicAdd(P.done + slot, 1u) + 1u == rp->items ? 1u : 0u;
      last = __shfl_sync(kFull, last, 0);
      if (last) {
        __threadfence();
        unsigned long long *res = P.host_res + 64ull * slot;
        for (int jj = (int)lane; jj < w; jj += 32) res[jj] = atomicExch(out + jj, 0ull);
        if (lane == 0) atomicExch(P.done + slot, 0u);
        __threadfence_system();
        __syncwarp();
        if (lane == 0) {
          __threadfence_system();
          *reinterpret_cast<volatile unsigned int *>(P.flags + slot) = rp->tag;
          __threadfence_system();
        }
      }
      // the run's record is read no more: one item fewer to count
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        atomicSub(&rp->left, 1u);
      }
    }
  }
  // leave: the last warp out resets the launch state for the next launch
  __syncwarp();
  if (lane == 0) {
    const unsigned total = gridDim.x * WPB;
    if (atomicAdd(&st->exited, 1u) == total - 1u) {
      __threadfence();
      *reinterpret_cast<volatile unsigned long long *>(&st->head) =
          *reinterpret_cast<volatile unsigned long long *>(&st->tickets);
      *reinterpret_cast<volatile unsigned int *>(&st->stop) = 0u;
      *reinterpret_cast<volatile unsigned int *>(&st->exited) = 0u;
      __threadfence();
    }
  }
}

#define POSPOP_RES(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&resident_kernel<BS, MINB, D, H>), BS, MINB, D, H}

static const Variant kResident[] = {POSPOP_FAMILY(POSPOP_RES)};

int resident_variant_count() { return (int)(sizeof(kResident) / sizeof(kResident[0])); }
const Variant &resident_variant(int i) { return kResident[i]; }

}  // namespace pospop

// pospop_batch.cuh -- batched counting over many arrays: planning kernels
// (work items per array, prefix sums) and the persistent counting kernel.
// Templated on the array source: CSR byte offsets from one base with one w
// (pospopcnt_batch), or gathered regions all counted into one counter array
// (pospopcnt_gather).
#pragma once

#include <cstdint>

#include "pospop_device.cuh"
#include "pospop_internal.h"

namespace pospop {

// Byte range [s, e) of array a, its width and its output counters.
struct ArrayRef {
  uint64_t s, e;
  int w;
  unsigned long long *out;
};

template <int SRC>
__device__ __forceinline__ ArrayRef array_ref(const BatchParams &P, uint64_t a) {
  ArrayRef r;
  if (SRC == kSrcGather) {
    r.s = __ldg(P.gptrs + a);
    r.e = r.s + __ldg(P.glens + a);
    r.w = P.w;
    r.out = P.counts;
  } else {
    const uint64_t base = (uint64_t)P.base;
    r.s = base + __ldg(P.offsets + a);
    r.e = base + __ldg(P.offsets + a + 1);
    r.w = P.w;
    r.out = P.counts + a * (uint64_t)P.w;
  }
  return r;
}

// ---------------------------------------------------------------------------
// Planning.  Array a spans granules [s/16, ceil(e/16)); its rows of 32
// granules are cut into work items of item_rows[batch_class(rows)] rows.
// item_start is the exclusive prefix sum of the items per array.  Decreasing
// CSR offsets set the status and give the array no items.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t span_items(uint64_t s, uint64_t e,
                                               const uint32_t (&item_rows)[kBatchClasses]) {
  if (e <= s) return 0;
  const uint64_t G = (((e + 15u) & ~15ull) - (s & ~15ull)) >> 4;
  const uint64_t R = (G + 31u) >> 5;
  const uint32_t ir = item_rows[batch_class(R)];
  return (R + ir - 1) / ir;
}

// Inclusive block-wide scan of one value per thread (kPlanThreads threads).
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t *warp_tot) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(kFull, v, d);
    if ((int)lane >= d) v += t;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t t = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t u = __shfl_up_sync(kFull, t, d);
      if ((int)lane >= d) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (warp > 0) v += warp_tot[warp - 1];
  return v;
}

template <int SRC>
__global__ void __launch_bounds__(kPlanThreads) plan_items_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  pdl_enter();
  const uint64_t a0 = (uint64_t)blockIdx.x * kPlanChunk + (uint64_t)threadIdx.x * kPlanPerThread;
  uint64_t local = 0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kPlanPerThread; k++) {
    const uint64_t a = a0 + k;
    if (a < P.m) {
      uint64_t s, e;
      if (SRC == kSrcGather) {
        s = P.gptrs[a];
        e = s + P.glens[a];
      } else {
        const uint64_t o0 = P.offsets[a], o1 = P.offsets[a + 1];
        if (o1 < o0) bad = true;
        s = P.base_addr + o0;
        e = P.base_addr + o1;
      }
      const uint64_t it = span_items(s, e, P.item_rows);
      P.item_start[a] = it;
      local += it;
    }
  }
  if (bad) *P.status = -1;
  const uint64_t incl = block_inclusive_scan(local, red);
  if (threadIdx.x == kPlanThreads - 1) P.block_sum[blockIdx.x] = incl;
}

// ---------------------------------------------------------------------------
// Persistent counting.  Warps take runs of consecutive work items per
// atomic (guided: longer runs while much work is left), find the first
// item's array with a 32-way warp search over item_start, and look the
// run's other items up in a window of 32 arrays' metadata.  Each item is a
// contiguous run of rows of one array, counted with the per-thread
// algorithm and added to that array's counters.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t find_array(const uint64_t *__restrict__ item_start, uint64_t m,
                                               uint64_t i, unsigned lane) {
  // Largest a in [0, m) with item_start[a] <= i (item_start[0] = 0 <= i < item_start[m]).
  uint64_t lo = 0, hi = m;
  while (hi - lo > 1) {
    const uint64_t span = hi - lo;
    const uint64_t idx = lo + span * (lane + 1) / 33;
    const bool le = __ldg(item_start + idx) <= i;
    const unsigned b = __ballot_sync(kFull, le);
    const int c = __popc(b);
    const uint64_t nlo = c > 0 ? lo + span * (uint64_t)c / 33 : lo;
    const uint64_t nhi = c < 32 ? lo + span * (uint64_t)(c + 1) / 33 : hi;
    lo = nlo;
    hi = nhi > lo ? nhi : lo + 1;
  }
  return lo;
}

constexpr uint64_t kMaxGrab = 8;    // work items per grab, at most

// PAR2: w = 256, where a word spans two granules (the two-parity flush).
template <int SRC, int BS, int MINB, int DEPTH, int HINT, bool PAR2 = false>
__global__ void __launch_bounds__(BS, MINB) batch_kernel(BatchParams P) {
  // Gathered regions all add into one counter array: accumulate per block in
  // shared memory, one atomic per counter per block at the end.
  constexpr int kAcc = SRC == kSrcGather ? (PAR2 ? 256 : 128) : 1;
  __shared__ unsigned long long gacc[kAcc];
  pdl_enter();
  if (SRC == kSrcGather) {
    for (int j = threadIdx.x; j < kAcc; j += BS) gacc[j] = 0ull;
    __syncthreads();
  }
  if (*P.status != 0) return;   // planning rejected the offsets: change nothing
  const unsigned lane = threadIdx.x & 31u;
  const Xpose xk = make_xpose(lane);
  const uint64_t total = P.item_start[P.m];
  // Guided self-scheduling: a grab takes about 1/(4 TW) of the items left
  // (at least P.grab, at most kMaxGrab), so early grabs are runs of
  // consecutive items (one array search per run, then a forward walk) and
  // late grabs are short (balance at the end).  The next grab is requested
  // before the current items are counted, so the atomic's round trip
  // overlaps the counting.  Measured on GB300 against one item per grab: a
  // batch of 200000 arrays of 1..1536 B 32% faster, 100000 gathered regions
  // 0.7% faster, the 55 GB ragged batch unchanged (factor 8 or a cap of 16
  // or 64 items: the tiny batch gains less or the large batches lose).
  const uint64_t TW = (uint64_t)gridDim.x * (BS / 32);
  auto grab_size = [&](uint64_t seen) -> unsigned long long {
    const uint64_t left = total > seen ? total - seen : 0;
    uint64_t g = left / (4 * TW);
    if (g < P.grab) g = P.grab;
    return g < kMaxGrab ? g : kMaxGrab;
  };
  unsigned long long nxt = 0, nxt_g = 0;
  if (lane == 0) {
    nxt_g = grab_size(0);
    nxt = atomicAdd(P.next, nxt_g);
  }
  for (;;) {
    const unsigned long long i0 = __shfl_sync(kFull, nxt, 0);
    const unsigned long long g = __shfl_sync(kFull, nxt_g, 0);
    if (i0 >= total) break;
    if (lane == 0) {
      nxt_g = grab_size(i0 + g);
      nxt = atomicAdd(P.next, nxt_g);
    }
    uint64_t a = find_array(P.item_start, P.m, i0, lane);
    const uint64_t i1 = (i0 + g < total) ? i0 + g : total;
    // Metadata window: lane j holds item_start and the start (and, gathered,
    // the length) of array a + j, read by one warp-wide load each, so the
    // grab's items find their arrays with a ballot instead of a chain of
    // dependent loads per item (arrays a .. a + 30 are covered; an item of a
    // later array takes the per-item loads).
    const uint64_t a_win = a;
    const uint64_t wj = a_win + lane;
    const uint64_t win_start = wj <= P.m ? __ldg(P.item_start + wj) : ~0ull;
    uint64_t win_lo = 0, win_len = 0;
    if (wj <= P.m) {
      if (SRC == kSrcGather) {
        if (wj < P.m) {
          win_lo = __ldg(P.gptrs + wj);
          win_len = __ldg(P.glens + wj);
        }
      } else {
        win_lo = __ldg(P.offsets + wj);
      }
    }
    for (uint64_t i = i0; i < i1; i++) {
      const unsigned in = __ballot_sync(kFull, win_start <= i);
      const int j = __popc(in) - 1;   // window arrays with item_start <= i form a prefix
      ArrayRef r;
      uint64_t k;
      if (j < 31) {
        a = a_win + (uint64_t)j;
        k = i - __shfl_sync(kFull, win_start, j);
        const uint64_t lo = __shfl_sync(kFull, win_lo, j);
        if (SRC == kSrcGather) {
          r.s = lo;
          r.e = lo + __shfl_sync(kFull, win_len, j);
          r.out = P.counts;
        } else {
          const uint64_t hi = __shfl_sync(kFull, win_lo, j + 1);
          r.s = (uint64_t)P.base + lo;
          r.e = (uint64_t)P.base + hi;
          r.out = P.counts + a * (uint64_t)P.w;
        }
        r.w = P.w;
      } else {
        while (__ldg(P.item_start + a + 1) <= i) a++;
        k = i - __ldg(P.item_start + a);
        r = array_ref<SRC>(P, a);
      }
      Span s;
      const uint64_t A = r.s & ~15ull;
      s.A = reinterpret_cast<const uint8_t *>(A);
      s.head = (uint32_t)(r.s - A);
      s.G = (((r.e + 15u) & ~15ull) - A) >> 4;
      s.tail = (uint32_t)(r.e - (A + 16u * (s.G - 1)));
      const uint32_t rot = (8u * s.head) & (uint32_t)(r.w - 1);
      const uint64_t R = span_rows(s);
      const uint32_t ir = P.item_rows[batch_class(R)];
      const uint64_t r0 = k * ir;
      const uint64_t r1 = (r0 + ir < R) ? r0 + ir : R;
      unsigned long long *out = r.out;
      if (!PAR2 && P.regroup && r.w == 8 && r1 - r0 <= 3) {
        uint32_t lo = 0u, hi = 0u;
        regroup_rows_w8(s, r0, 1, r1 - r0, lane, PlainLoader<HINT>{}, lo, hi);
        if (SRC == kSrcGather)
          regroup_emit_w8(lo, hi, lane, [&](uint32_t j, unsigned long long v) {
            if (v) atomicAdd(&gacc[j], v);
          });
        else
          regroup_emit_w8(lo, hi, lane, [&](uint32_t j, unsigned long long v) {
            if (v) atomicAdd(out + j, v);
          });
        continue;
      }
      uint32_t cnt[4] = {0u, 0u, 0u, 0u};
      uint32_t cnt_odd[4] = {0u, 0u, 0u, 0u};
      // an item starts at an even granule (row r0 of a 16-byte-aligned span),
      // so lane parity is granule parity, as the two-parity flush requires
      count_rows<DEPTH, HINT, PlainLoader<HINT>, PAR2>(s, r0, 1, r1 - r0, lane, xk, cnt,
                                                       PlainLoader<HINT>{}, cnt_odd);
      auto to_gacc = [&](uint32_t j, unsigned long long v) {
        if (v) atomicAdd(&gacc[j], v);
      };
      auto to_out = [&](uint32_t j, unsigned long long v) {
        if (v) atomicAdd(out + j, v);
      };
      if (PAR2) {
        if (SRC == kSrcGather)
          fold_counts_256(cnt, cnt_odd, rot, lane, to_gacc);
        else
          fold_counts_256(cnt, cnt_odd, rot, lane, to_out);
      } else {
        if (SRC == kSrcGather)
          fold_counts(cnt, r.w, rot, lane, to_gacc);
        else
          fold_counts(cnt, r.w, rot, lane, to_out);
      }
    }
  }
  if (SRC == kSrcGather) {
    __syncthreads();
    for (int j = threadIdx.x; j < P.w; j += BS)
      if (gacc[j]) atomicAdd(P.counts + j, gacc[j]);
  }
}

// w = 256 variants: the tune table's launch shapes, flush depth 16.
#define POSPOP_FAMILY256(M) M(512, 1, 16, 0), M(512, 1, 16, 1), M(256, 2, 16, 1), M(128, 4, 16, 1)

#define POSPOP_FAMILY(M)                                                  \
  M(256, 2, 16, 0), M(256, 2, 16, 1), M(256, 2, 32, 0), M(256, 2, 32, 1), \
  M(512, 1, 16, 0), M(512, 1, 16, 1), M(512, 1, 32, 0), M(512, 1, 32, 1), \
  M(128, 4, 16, 0), M(128, 4, 16, 1), M(128, 4, 32, 0), M(128, 4, 32, 1)

}  // namespace pospop

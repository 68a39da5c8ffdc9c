// pospop_batch.cu -- the sm_103a batched positional population count:
// planning kernels over CSR offsets and the persistent counting kernel.
//
// The per-thread algorithm is the paper's (arXiv 2412.16370, Section 4:
// CSA_15 head reduction, CSA_16+4 main loop, a16 accumulation, final
// accumulation, tail, fold f_w); the GPU decomposition is this library's:
// rows of 32 granules per warp, warp-transpose popcounts, a block reduction
// in shared memory and one 64-bit atomic per counter per block.
#include <cstdint>

#include "pospop_device.cuh"
#include "pospop_internal.h"

namespace pospop {

__device__ __forceinline__ Span to_span(const SpanH &h) {
  Span s;
  s.A = h.A;
  s.G = h.G;
  s.head = h.head;
  s.tail = h.tail;
  return s;
}

// ---------------------------------------------------------------------------
// Batched: planning.  Array a spans granules [start/16, ceil(end/16)); its
// rows are cut into work items of item_rows rows.  item_start is the
// exclusive prefix sum of the items per array; decreasing offsets set the
// status and give the array no items.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t array_items(uint64_t base, uint64_t o0, uint64_t o1,
                                                uint32_t item_rows) {
  if (o1 <= o0) return 0;
  const uint64_t s = base + o0, e = base + o1;
  const uint64_t G = (((e + 15u) & ~15ull) - (s & ~15ull)) >> 4;
  const uint64_t R = (G + 31u) >> 5;
  return (R + item_rows - 1) / item_rows;
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

__global__ void __launch_bounds__(kPlanThreads) plan_items_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  const uint64_t a0 = (uint64_t)blockIdx.x * kPlanChunk + (uint64_t)threadIdx.x * kPlanPerThread;
  uint64_t local = 0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kPlanPerThread; k++) {
    const uint64_t a = a0 + k;
    if (a < P.m) {
      const uint64_t o0 = P.offsets[a], o1 = P.offsets[a + 1];
      if (o1 < o0) bad = true;
      const uint64_t it = array_items(P.base_addr, o0, o1, P.item_rows);
      P.item_start[a] = it;
      local += it;
    }
  }
  if (bad) *P.status = -1;
  const uint64_t incl = block_inclusive_scan(local, red);
  if (threadIdx.x == kPlanThreads - 1) P.block_sum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kPlanThreads) plan_scan_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < P.nblocks; b0 += kPlanThreads) {
    const uint32_t b = b0 + threadIdx.x;
    const uint64_t v = b < P.nblocks ? P.block_sum[b] : 0;
    const uint64_t incl = block_inclusive_scan(v, red);
    const uint64_t c = carry;
    if (b < P.nblocks) P.block_sum[b] = c + incl - v;   // exclusive
    __syncthreads();
    if (threadIdx.x == kPlanThreads - 1) carry = c + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.item_start[P.m] = carry;
    *P.next = 0ull;
  }
}

__global__ void __launch_bounds__(kPlanThreads) plan_apply_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  const uint64_t a0 = (uint64_t)blockIdx.x * kPlanChunk + (uint64_t)threadIdx.x * kPlanPerThread;
  uint64_t it[kPlanPerThread];
  uint64_t local = 0;
#pragma unroll
  for (int k = 0; k < kPlanPerThread; k++) {
    it[k] = (a0 + k < P.m) ? P.item_start[a0 + k] : 0;
    local += it[k];
  }
  const uint64_t incl = block_inclusive_scan(local, red);
  uint64_t run = P.block_sum[blockIdx.x] + incl - local;
#pragma unroll
  for (int k = 0; k < kPlanPerThread; k++) {
    if (a0 + k < P.m) P.item_start[a0 + k] = run;
    run += it[k];
  }
}

// ---------------------------------------------------------------------------
// Batched: persistent counting.  Warps take `grab` consecutive work items
// per atomic, find the first item's array with a 32-way warp search over
// item_start, then walk forward.  Each item is a contiguous run of rows of
// one array, counted with the per-thread algorithm and added to that
// array's counters.
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

template <int BS, int MINB, int DEPTH, int HINT>
__global__ void __launch_bounds__(BS, MINB) batch_kernel(BatchParams P) {
  if (*P.status != 0) return;   // planning rejected the offsets: change nothing
  const unsigned lane = threadIdx.x & 31u;
  const Xpose xk = make_xpose(lane);
  const uint64_t total = P.item_start[P.m];
  const uint64_t base = (uint64_t)P.base;
  for (;;) {
    unsigned long long i0 = 0;
    if (lane == 0) i0 = atomicAdd(P.next, (unsigned long long)P.grab);
    i0 = __shfl_sync(kFull, i0, 0);
    if (i0 >= total) break;
    uint64_t a = find_array(P.item_start, P.m, i0, lane);
    const uint64_t i1 = (i0 + P.grab < total) ? i0 + P.grab : total;
    for (uint64_t i = i0; i < i1; i++) {
      while (__ldg(P.item_start + a + 1) <= i) a++;
      const uint64_t k = i - __ldg(P.item_start + a);
      const uint64_t s0 = base + __ldg(P.offsets + a), e0 = base + __ldg(P.offsets + a + 1);
      Span s;
      const uint64_t A = s0 & ~15ull;
      s.A = reinterpret_cast<const uint8_t *>(A);
      s.head = (uint32_t)(s0 - A);
      s.G = (((e0 + 15u) & ~15ull) - A) >> 4;
      s.tail = (uint32_t)(e0 - (A + 16u * (s.G - 1)));
      const uint32_t rot = (8u * s.head) & (uint32_t)(P.w - 1);
      const uint64_t R = span_rows(s);
      const uint64_t r0 = k * P.item_rows;
      const uint64_t r1 = (r0 + P.item_rows < R) ? r0 + P.item_rows : R;
      uint32_t cnt[4] = {0u, 0u, 0u, 0u};
      count_rows<DEPTH, HINT>(s, r0, 1, r1 - r0, lane, xk, cnt);
      unsigned long long *out = P.counts + a * (uint64_t)P.w;
      fold_counts(cnt, P.w, rot, lane, [&](uint32_t j, unsigned long long v) {
        if (v) atomicAdd(out + j, v);
      });
    }
  }
}

// ---------------------------------------------------------------------------
// Variant table (every variant fits 128 registers per thread, no spills).
// ---------------------------------------------------------------------------
#define POSPOP_BV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&batch_kernel<BS, MINB, D, H>), BS, MINB, D, H}
#define POSPOP_FAMILY(M)                                                  \
  M(256, 2, 16, 0), M(256, 2, 16, 1), M(256, 2, 32, 0), M(256, 2, 32, 1), \
  M(512, 1, 16, 0), M(512, 1, 16, 1), M(512, 1, 32, 0), M(512, 1, 32, 1), \
  M(128, 4, 16, 0), M(128, 4, 16, 1), M(128, 4, 32, 0), M(128, 4, 32, 1)

static const Variant kBatch[] = {POSPOP_FAMILY(POSPOP_BV)};

int batch_variant_count() { return (int)(sizeof(kBatch) / sizeof(kBatch[0])); }
const Variant &batch_variant(int i) { return kBatch[i]; }

const void *plan_items_fn() { return reinterpret_cast<const void *>(&plan_items_kernel); }
const void *plan_scan_fn() { return reinterpret_cast<const void *>(&plan_scan_kernel); }
const void *plan_apply_fn() { return reinterpret_cast<const void *>(&plan_apply_kernel); }

}  // namespace pospop

// pospop_multi.cu -- several large counts in one launch (pospopcnt_multi
// for groups of large counts): the single-array kernel's grid-stride row
// schedule, run over the rows of every count of the group in turn.
//
// The per-thread algorithm is the paper's (arXiv 2412.16370, Section 4), as
// in pospop_stream.cu; only the schedule over several counts is new.
#include <cstdint>

#include "pospop_batch.cuh"

namespace pospop {

// ---------------------------------------------------------------------------
// Several large counts in one grid-stride launch (pospopcnt_multi for groups
// of large counts).  The counts' rows form one sequence (count 0's rows, then
// count 1's, ...) and warp gw of NW takes the sequence's rows gw, gw + NW,
// ..., so within each count the warps read rows with stride NW exactly as
// stream_kernel does, and the group pays one launch ramp and one tail
// instead of one per count.  Per count, the warps' folded counters meet in
// shared memory and one atomic per counter per block adds them to that
// count's counters (the count loop is uniform over the block).  The host
// skips empty counts, bounds the rows per warp as for a single array and
// keeps every count below 2^32 rows.
// ---------------------------------------------------------------------------
template <int BS, int MINB, int DEPTH, int HINT>
__global__ void __launch_bounds__(BS, MINB)
    multi_stream_kernel(const __grid_constant__ ServeParams P) {
  __shared__ unsigned long long acc[64];
  pdl_enter();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = threadIdx.x >> 5;
  if (threadIdx.x < 64) acc[threadIdx.x] = 0ull;
  __syncthreads();
  constexpr unsigned WPB = BS / 32;
  // 32-bit index arithmetic (a 64-bit division is a call, and its register
  // traffic would spill the CSA state): the host keeps NW and every count's
  // rows below 2^32 and passes, in req[k].items, the position of count k's
  // row 0 in the group's row sequence modulo NW
  const uint32_t NW = gridDim.x * WPB;
  const uint32_t gw = blockIdx.x * WPB + warp;
  const Xpose xk = make_xpose(lane);
#pragma unroll 1
  for (uint32_t k = 0; k < P.n; k++) {
    const ServeReq &rq = P.req[k];
    const uint64_t s0 = (uint64_t)rq.ptr, e0 = s0 + rq.nbytes;
    Span s;
    const uint64_t A = s0 & ~15ull;
    s.A = reinterpret_cast<const uint8_t *>(A);
    s.head = (uint32_t)(s0 - A);
    s.G = (((e0 + 15u) & ~15ull) - A) >> 4;
    s.tail = (uint32_t)(e0 - (A + 16u * (s.G - 1)));
    const uint32_t rot = (8u * s.head) & (uint32_t)(rq.w - 1);
    const uint32_t R = (uint32_t)span_rows(s);
    // this warp's rows of count k: the r with (first + r) mod NW == gw
    const uint32_t first_mod = rq.items;
    const uint32_t r0 = gw >= first_mod ? gw - first_mod : gw + (NW - first_mod);
    const uint32_t mine = R > r0 ? (R - r0 - 1) / NW + 1 : 0;
    if (mine > 0) {   // warp-uniform
      uint32_t cnt[4] = {0u, 0u, 0u, 0u};
      count_rows<DEPTH, HINT>(s, r0, NW, mine, lane, xk, cnt, PlainLoader<HINT>{});
      fold_counts(cnt, rq.w, rot, lane, [&](uint32_t j, unsigned long long v) {
        if (v) atomicAdd(&acc[j], v);
      });
    }
    __syncthreads();
    if ((int)threadIdx.x < rq.w) {
      const unsigned long long v = acc[threadIdx.x];
      if (v) atomicAdd(rq.out + threadIdx.x, v);
      acc[threadIdx.x] = 0ull;
    }
    __syncthreads();
  }
}

// Variants: the single-array family's launch shapes, in its order (so the
// single-array tune entry's index picks the same shape here).
#define POSPOP_MSV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&multi_stream_kernel<BS, MINB, D, H>), BS, MINB, D, H}
static const Variant kMultiStream[] = {POSPOP_FAMILY(POSPOP_MSV)};

int multi_stream_variant_count() { return (int)(sizeof(kMultiStream) / sizeof(kMultiStream[0])); }
const Variant &multi_stream_variant(int i) { return kMultiStream[i]; }

}  // namespace pospop

// pospop_select.cu -- the single-array count restricted to selected words
// (pospopcnt_masked): Fig. 2's loop over only the words whose bit is set in
// a selection bitmap, i.e. the GROUP BY count of Section 1 with a WHERE
// filter.  Same row schedule, CSA networks, transpose flush and reductions as
// stream_kernel; every granule is ANDed with its words' selection bits
// (expanded to byte masks) before it enters the CSA network.
#include <cstdint>

#include "pospop_batch.cuh"

namespace pospop {

template <int BS, int MINB, int DEPTH, int HINT, int WLOG>
__global__ void __launch_bounds__(BS, MINB) select_kernel(SelectParams Q) {
  __shared__ unsigned long long acc[64];
  pdl_enter();
  const StreamParams &P = Q.sp;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = threadIdx.x >> 5;
  if (threadIdx.x < 64) acc[threadIdx.x] = 0ull;
  __syncthreads();

  constexpr unsigned WPB = BS / 32;
  const uint64_t NW = (uint64_t)gridDim.x * WPB;
  const uint64_t gw = (uint64_t)blockIdx.x * WPB + warp;
  const uint64_t nr = P.row_end - P.row_begin;
  const uint64_t mine = nr > gw ? (nr - gw + NW - 1) / NW : 0;

  Span s;
  s.A = P.s.A;
  s.G = P.s.G;
  s.head = P.s.head;
  s.tail = P.s.tail;
  SelectLoader<HINT, WLOG> ld;
  ld.m = Selection{Q.bits, Q.nbits, Q.nbytes, P.s.head >> WLOG};
  const Xpose xk = make_xpose(lane);
  uint32_t cnt[4] = {0u, 0u, 0u, 0u};
  count_rows<DEPTH, HINT>(s, P.row_begin + gw, NW, mine, lane, xk, cnt, ld);
  fold_counts(cnt, P.w, P.rot, lane, [&](uint32_t j, unsigned long long v) {
    if (v) atomicAdd(&acc[j], v);
  });
  __syncthreads();
  if ((int)threadIdx.x < P.w) {
    const unsigned long long v = acc[threadIdx.x];
    if (v) atomicAdd(&P.counts[threadIdx.x], v);
  }
}

// Variants: the launch shapes the tune table uses (flush depth 16), each
// specialised for the four word sizes; index = 4 * shape + log2(W).
#define POSPOP_SELV(BS, MINB, H, WL) \
  Variant{reinterpret_cast<const void *>(&select_kernel<BS, MINB, 16, H, WL>), BS, MINB, 16, H}
#define POSPOP_SEL4(BS, MINB, H) \
  POSPOP_SELV(BS, MINB, H, 0), POSPOP_SELV(BS, MINB, H, 1), POSPOP_SELV(BS, MINB, H, 2), \
      POSPOP_SELV(BS, MINB, H, 3)

static const Variant kSelect[] = {POSPOP_SEL4(512, 1, 0), POSPOP_SEL4(512, 1, 1),
                                  POSPOP_SEL4(256, 2, 1), POSPOP_SEL4(128, 4, 1)};

int select_variant_count() { return (int)(sizeof(kSelect) / sizeof(kSelect[0])); }
const Variant &select_variant(int i) { return kSelect[i]; }

}  // namespace pospop

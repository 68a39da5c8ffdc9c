// pospop_stream.cu -- the sm_103a single-array kernel of the positional
// population count.
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
// Single array.  Warp gw of NW takes rows row_begin + gw, + NW, + 2NW, ...
// so that at any moment the grid streams one contiguous region.  Per block,
// the warps' folded counters meet in shared memory; one atomic per counter
// per block adds them to the caller's counts (step 8, f_w(C, c)).
// ---------------------------------------------------------------------------
template <int BS, int MINB, int DEPTH, int HINT, bool PAR2 = false>
__global__ void __launch_bounds__(BS, MINB) stream_kernel(StreamParams P) {
  __shared__ unsigned long long acc[256];
  pdl_enter();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < 256; j += BS) acc[j] = 0ull;
  __syncthreads();

  constexpr unsigned WPB = BS / 32;
  const uint64_t NW = (uint64_t)gridDim.x * WPB;
  const uint64_t gw = (uint64_t)blockIdx.x * WPB + warp;
  const uint64_t nr = P.row_end - P.row_begin;
  const uint64_t mine = nr > gw ? (nr - gw + NW - 1) / NW : 0;

  const Xpose xk = make_xpose(lane);
  auto to_shared = [&](uint32_t j, unsigned long long v) {
    if (v) atomicAdd(&acc[j], v);
  };
  if (!PAR2 && P.regroup && P.w == 8 && mine <= 3) {   // warp-uniform choice
    uint32_t lo = 0u, hi = 0u;
    regroup_rows_w8(to_span(P.s), P.row_begin + gw, NW, mine, lane, PlainLoader<HINT>{}, lo, hi);
    regroup_emit_w8(lo, hi, lane, to_shared);
  } else {
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    uint32_t cnt_odd[4] = {0u, 0u, 0u, 0u};
    count_rows<DEPTH, HINT, PlainLoader<HINT>, PAR2>(to_span(P.s), P.row_begin + gw, NW, mine,
                                                     lane, xk, cnt, PlainLoader<HINT>{}, cnt_odd);
    if (PAR2)
      fold_counts_256(cnt, cnt_odd, P.rot, lane, to_shared);
    else
      fold_counts(cnt, P.w, P.rot, lane, to_shared);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < P.w; j += BS) {
    const unsigned long long v = acc[j];
    if (v) atomicAdd(&P.counts[j], v);
  }
}

// ---------------------------------------------------------------------------
// Variant tables (every variant fits 128 registers per thread, no spills).
// ---------------------------------------------------------------------------
#define POSPOP_SV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&stream_kernel<BS, MINB, D, H>), BS, MINB, D, H}
#define POSPOP_FAMILY(M)                                                  \
  M(256, 2, 16, 0), M(256, 2, 16, 1), M(256, 2, 32, 0), M(256, 2, 32, 1), \
  M(512, 1, 16, 0), M(512, 1, 16, 1), M(512, 1, 32, 0), M(512, 1, 32, 1), \
  M(128, 4, 16, 0), M(128, 4, 16, 1), M(128, 4, 32, 0), M(128, 4, 32, 1)

static const Variant kStream[] = {POSPOP_FAMILY(POSPOP_SV)};

// w = 256 (two-parity flush): the tune table's launch shapes, flush depth 16.
#define POSPOP_SV256(BS, MINB, H) \
  Variant{reinterpret_cast<const void *>(&stream_kernel<BS, MINB, 16, H, true>), BS, MINB, 16, H}
static const Variant kStream256[] = {POSPOP_SV256(512, 1, 0), POSPOP_SV256(512, 1, 1),
                                     POSPOP_SV256(256, 2, 1), POSPOP_SV256(128, 4, 1)};

int stream_variant_count() { return (int)(sizeof(kStream) / sizeof(kStream[0])); }
int stream256_variant_count() { return (int)(sizeof(kStream256) / sizeof(kStream256[0])); }
const Variant &stream256_variant(int i) { return kStream256[i]; }
const Variant &stream_variant(int i) { return kStream[i]; }

}  // namespace pospop

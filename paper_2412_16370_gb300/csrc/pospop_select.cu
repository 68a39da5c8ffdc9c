// pospop_select.cu -- the single-array count restricted to selected words
// (pospopcnt_masked): Fig. 2's loop over only the words whose bit is set in
// a selection bitmap, i.e. the GROUP BY count of Section 1 with a WHERE
// filter.  Same row schedule, CSA networks, transpose flush and reductions as
// stream_kernel; every granule is ANDed with its words' selection bits
// (expanded to byte masks) before it enters the CSA network.
#include <cstdint>

#include "pospop_batch.cuh"
#include "pospop_bulk.cuh"
#include "pospopcnt.h"

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

// ---------------------------------------------------------------------------
// Staged form.  The selected
// count does about half again the plain count's arithmetic per byte, so with
// its loads in registers a warp issues the next group's loads late and DRAM
// idles.  Here the copy engine keeps the bytes in flight instead: each warp
// owns a ring of S stages in shared memory, one CSA group (16 rows, 8 KiB of
// words) plus its 64 * CNT bytes of selection bits per stage, both filled by
// bulk copies (cp.async.bulk) that complete one mbarrier phase.  Chunk c is
// rows 16c .. 16c + 15; warps take chunks c = chunk0 + gw, + TW, ... below
// Q.nstaged (chunks wholly inside the span: chunk 0 only when the span
// starts on a 16-byte boundary and the bitmap on a 16-byte boundary), and
// warp 0 counts the remaining rows with count_rows.  Chunk c's selection
// bits start at bit sel_bit0 + 512 * CNT * c of the bitmap's 16-byte-aligned
// base, so the copy takes the 16-byte blocks around them (one block more
// when they do not start on a block) and every chunk's bits sit at the same
// offset in the stage.
// ---------------------------------------------------------------------------
template <int WLOG>
__host__ __device__ constexpr uint32_t staged_stage_bytes() {
  return kBulkChunk + 64u * (16u >> WLOG) + 16u;
}

template <int NW, int S, int WLOG>
constexpr int staged_smem() {
  return NW * S * (int)staged_stage_bytes<WLOG>() + NW * S * 8;
}

template <int NW, int S, int WLOG>
__global__ void __launch_bounds__(NW * 32, 1) select_staged_kernel(SelectParams Q) {
  constexpr uint32_t CNT = 16u >> WLOG;                // selection bits per granule
  constexpr uint32_t kStage = staged_stage_bytes<WLOG>();  // 16-byte multiple
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ unsigned long long acc[64];
  pdl_enter();
  const StreamParams &P = Q.sp;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x < 64) acc[threadIdx.x] = 0ull;
  __syncthreads();

  uint8_t *ring = smem + (size_t)warp * S * kStage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NW * S * kStage) + warp * S;
  const uint64_t TW = (uint64_t)gridDim.x * NW;
  const uint64_t gw = (uint64_t)blockIdx.x * NW + warp;
  const uint64_t nch = Q.nstaged;
  Span s;
  s.A = P.s.A;
  s.G = P.s.G;
  s.head = P.s.head;
  s.tail = P.s.tail;
  const Xpose xk = make_xpose(lane);
  uint32_t cnt[4] = {0u, 0u, 0u, 0u};

  const uint32_t h = P.s.head >> WLOG;                // words before the start in granule 0
  // bit offset of a chunk's bits in its copy (512 * CNT is a multiple of 128)
  const uint32_t sel_off = (uint32_t)((uint64_t)Q.sel_bit0 & 127u);
  auto fill = [&](int k, uint64_t c) {   // lane 0 only
    const uint32_t bar = smem_addr(bars + k);
    mbar_expect(bar, kBulkChunk + Q.sel_bytes);
    bulk_copy_tx(smem_addr(ring + k * kStage), s.A + c * kBulkChunk, kBulkChunk, bar);
    const uint64_t first_bit = (uint64_t)((int64_t)(c * (512u * CNT)) + Q.sel_bit0);
    bulk_copy_tx(smem_addr(ring + k * kStage + kBulkChunk), Q.sel_base + (first_bit >> 7) * 16u,
                 Q.sel_bytes, bar);
  };
  const uint64_t c0 = Q.chunk0 + gw;
  if (lane == 0) {
    for (int k = 0; k < S; k++) mbar_init(smem_addr(bars + k));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < S; k++)
      if (c0 + (uint64_t)k * TW < nch) fill(k, c0 + (uint64_t)k * TW);
  }
  __syncwarp();

  Planes p;
  p.a1 = p.a2 = p.a4 = p.a8 = v4_zero();
  uint64_t it = 0;
  bool timed_out = false;
  for (uint64_t c = c0; c < nch; c += TW, it++) {
    const int k = (int)(it % S);
    if (!__all_sync(kFull,
                    mbar_wait(smem_addr(bars + k), (uint32_t)((it / S) & 1u), Q.wait_cycles))) {
      timed_out = true;
      break;
    }
    const uint4 *d = reinterpret_cast<const uint4 *>(ring + k * kStage);
    const uint32_t *sel = reinterpret_cast<const uint32_t *>(ring + k * kStage + kBulkChunk);
    V4 v[16];
#pragma unroll
    for (int r = 0; r < 16; r++) {
      const uint4 x = d[r * 32 + lane];
      v[r] = V4{{x.x, x.y, x.z, x.w}};
      const uint32_t bit = sel_off + (uint32_t)(r * 32 + lane) * CNT;
      const uint32_t sh = bit & 31u;
      // a window straddles into the next word only when the chunk's bit
      // offset is not a multiple of CNT; that word's bits then lie inside
      // the copy
      const uint32_t w1 = (sh + CNT > 32u) ? sel[(bit >> 5) + 1] : 0u;
      apply_selection<WLOG>(v[r], __funnelshift_r(sel[bit >> 5], w1, sh));
    }
    __syncwarp();   // every lane has read the stage before it is refilled
    const uint64_t nx = c + (uint64_t)S * TW;
    if (lane == 0 && nx < nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fill(k, nx);
    }
    flush_plane<4>(cnt, csa16(p, v), xk);
  }
  if (timed_out) {
    // report, then wait (bounded by the fixed kBulkWaitCycles, whatever
    // Q.wait_cycles is) for this warp's copies still in flight so that none
    // lands after the block has left; the block still meets at the barrier
    // below
    if (lane == 0 && Q.status) atomicExch(Q.status, POSPOP_ETIMEDOUT);
    for (uint64_t j = 0, c = c0 + it * TW; j < (uint64_t)S && c < nch; j++, c += TW)
      (void)mbar_wait(smem_addr(bars + (int)((it + j) % S)), (uint32_t)(((it + j) / S) & 1u));
  }
  // final accumulation of the staged chunks (Section 4.5)
  flush_plane<3>(cnt, p.a8, xk);
  flush_plane<2>(cnt, p.a4, xk);
  flush_plane<1>(cnt, p.a2, xk);
  flush_plane<0>(cnt, p.a1, xk);
  // rows outside the staged chunks: the span's start (chunk 0 when the
  // span starts inside a granule) and end (partial granule, rows past the
  // last staged group)
  if (gw == 0) {
    SelectLoader<0, WLOG> ld;
    ld.m = Selection{Q.bits, Q.nbits, Q.nbytes, h};
    const uint64_t R = span_rows(s);
    if (Q.chunk0 > 0) count_rows<16, 0>(s, 0, 1, 16u * Q.chunk0, lane, xk, cnt, ld);
    const uint64_t r0 = 16u * nch;
    if (R > r0) count_rows<16, 0>(s, r0, 1, R - r0, lane, xk, cnt, ld);
  }
  fold_counts(cnt, P.w, P.rot, lane, [&](uint32_t j, unsigned long long v) {
    if (v) atomicAdd(&acc[j], v);
  });
  __syncthreads();
  if ((int)threadIdx.x < P.w) {
    const unsigned long long v = acc[threadIdx.x];
    if (v) atomicAdd(&P.counts[threadIdx.x], v);
  }
}

// Ring shapes (warps per block, stages per warp), each for the four word
// sizes; index = 4 * shape + log2(W).  `depth` records the stages.
#define POSPOP_SELS(NW, S, WL)                                                          \
  Variant{reinterpret_cast<const void *>(&select_staged_kernel<NW, S, WL>), NW * 32, 1, S, \
          0, staged_smem<NW, S, WL>()}
#define POSPOP_SELS4(NW, S) \
  POSPOP_SELS(NW, S, 0), POSPOP_SELS(NW, S, 1), POSPOP_SELS(NW, S, 2), POSPOP_SELS(NW, S, 3)
static const Variant kSelectStaged[] = {POSPOP_SELS4(8, 3), POSPOP_SELS4(12, 2),
                                        POSPOP_SELS4(16, 1)};

int select_staged_variant_count() {
  return (int)(sizeof(kSelectStaged) / sizeof(kSelectStaged[0]));
}
const Variant &select_staged_variant(int i) { return kSelectStaged[i]; }

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

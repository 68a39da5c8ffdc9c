// pospop_roofline.cu -- the roofline read kernels (Section 5's "dummy"
// kernel: sum the input and add the sum to an output), the achievable-read
// reference for the counting kernels.
//
// Two ways to stream the same bytes:
//  * roofline_kernel: the counting kernel's own loads (one 16-byte
//    ld.global.nc per lane, 512-byte rows per warp, 16 rows in flight per
//    thread) and row schedule, with an add in place of the counting;
//  * roofline_bulk_kernel: the bytes are staged in shared memory by the
//    copy engine (cp.async.bulk, one-dimensional TMA, completion counted on
//    an mbarrier): each warp keeps a ring of S chunks of 8 KiB in flight and
//    sums a chunk from shared memory once its barrier phase completes.
// Both compute the exact sum of the 32-bit little-endian words.
#include <cstdint>

#include "pospop_bulk.cuh"
#include "pospop_device.cuh"
#include "pospop_internal.h"
#include "pospopcnt.h"

namespace pospop {

__device__ __forceinline__ unsigned long long sum_words(const V4 &v) {
  return (unsigned long long)v.x[0] + v.x[1] + (unsigned long long)v.x[2] + v.x[3];
}

// ---------------------------------------------------------------------------
// Direct loads.  Warp gw of NW reads rows gw, gw + NW, ... (rows of 32
// granules), 16 rows per step.
// ---------------------------------------------------------------------------
template <int BS, int HINT>
__global__ void __launch_bounds__(BS) roofline_kernel(RooflineParams P) {
  pdl_enter();
  constexpr unsigned WPB = BS / 32;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t NW = (uint64_t)gridDim.x * WPB;
  const uint64_t R = (P.G + 31) >> 5;
  const uint64_t Rfull = P.G >> 5;
  unsigned long long sum = 0;
  uint64_t row = (uint64_t)blockIdx.x * WPB + warp;
  for (; row + 15 * NW < Rfull; row += 16 * NW) {
    V4 v[16];
#pragma unroll
    for (int k = 0; k < 16; k++)
      v[k] = ldg_granule<HINT>(P.A + ((row + k * NW) * 32 + lane) * kGranule);
#pragma unroll
    for (int k = 0; k < 16; k++) sum += sum_words(v[k]);
  }
  for (; row < R; row += NW) {
    const uint64_t g = row * 32 + lane;
    if (g < P.G) sum += sum_words(ldg_granule<HINT>(P.A + g * kGranule));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
  if (lane == 0 && sum) atomicAdd(P.sum, sum);
}

// ---------------------------------------------------------------------------
// Bulk-copy staging.
// ---------------------------------------------------------------------------
template <int NW, int S>
__global__ void __launch_bounds__(NW * 32, 1) roofline_bulk_kernel(RooflineParams P) {
  extern __shared__ __align__(128) uint8_t smem[];
  pdl_enter();
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint8_t *ring = smem + (size_t)warp * S * kBulkChunk;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NW * S * kBulkChunk) + warp * S;
  const uint64_t TW = (uint64_t)gridDim.x * NW;
  const uint64_t gw = (uint64_t)blockIdx.x * NW + warp;
  const uint64_t nch = (P.G + 511) >> 9;
  // granules in chunk c (512 except for the last)
  auto granules = [&](uint64_t c) -> uint32_t {
    const uint64_t left = P.G - (c << 9);
    return (uint32_t)(left < 512 ? left : 512);
  };
  if (lane == 0) {
    for (int k = 0; k < S; k++) mbar_init(smem_addr(bars + k));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int k = 0; k < S; k++) {
      const uint64_t c = gw + (uint64_t)k * TW;
      if (c < nch)
        bulk_copy(smem_addr(ring + k * kBulkChunk), P.A + c * kBulkChunk, granules(c) * 16u,
                  smem_addr(bars + k));
    }
  }
  __syncwarp();
  unsigned long long sum = 0;
  uint64_t it = 0;
  bool timed_out = false;
  for (uint64_t c = gw; c < nch; c += TW, it++) {
    const int k = (int)(it % S);
    // warp-uniform: every lane leaves together if any lane's wait expired
    if (!__all_sync(kFull,
                    mbar_wait(smem_addr(bars + k), (uint32_t)((it / S) & 1u), P.wait_cycles))) {
      timed_out = true;
      break;
    }
    const uint32_t ng = granules(c);
    const uint4 *v = reinterpret_cast<const uint4 *>(ring + k * kBulkChunk);
#pragma unroll 4
    for (uint32_t g = lane; g < ng; g += 32) {
      const uint4 x = v[g];
      sum += (unsigned long long)x.x + x.y + (unsigned long long)x.z + x.w;
    }
    __syncwarp();   // every lane has read the stage before it is refilled
    const uint64_t nx = c + (uint64_t)S * TW;
    if (lane == 0 && nx < nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_copy(smem_addr(ring + k * kBulkChunk), P.A + nx * kBulkChunk, granules(nx) * 16u,
                smem_addr(bars + k));
    }
  }
  if (timed_out) {
    // report, then wait (bounded by the fixed kBulkWaitCycles, whatever
    // P.wait_cycles is) for this warp's copies still in flight so that none
    // lands after the block has left
    if (lane == 0 && P.status) atomicExch(P.status, POSPOP_ETIMEDOUT);
    for (uint64_t j = 0, c = gw + it * TW; j < (uint64_t)S && c < nch; j++, c += TW)
      (void)mbar_wait(smem_addr(bars + (int)((it + j) % S)), (uint32_t)(((it + j) / S) & 1u));
    return;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
  if (lane == 0 && sum) atomicAdd(P.sum, sum);
}

template <int NW, int S>
constexpr int bulk_smem() {
  return NW * S * (int)kBulkChunk + NW * S * 8;
}

// ---------------------------------------------------------------------------
// Variant table.  Load variant (hint) 0/1: direct loads without/with the L2
// 256-byte prefetch hint; 2: bulk-copy staging (dynamic shared memory).
// ---------------------------------------------------------------------------
#define POSPOP_RV(BS, H) \
  Variant{reinterpret_cast<const void *>(&roofline_kernel<BS, H>), BS, 1, 0, H, 0}
#define POSPOP_RB(NW, S)                                                                   \
  Variant{reinterpret_cast<const void *>(&roofline_bulk_kernel<NW, S>), NW * 32, 1, 0, 2, \
          bulk_smem<NW, S>()}

static const Variant kRoof[] = {POSPOP_RV(256, 0), POSPOP_RV(256, 1),  POSPOP_RV(512, 0),
                                POSPOP_RV(512, 1), POSPOP_RV(1024, 0), POSPOP_RV(1024, 1),
                                POSPOP_RB(8, 3),   POSPOP_RB(4, 3)};

int roofline_variant_count() { return (int)(sizeof(kRoof) / sizeof(kRoof[0])); }
const Variant &roofline_variant(int i) { return kRoof[i]; }

}  // namespace pospop

// pospop_batch.cu -- the sm_103a batched positional population count over
// CSR offsets (pospopcnt_batch): planning kernels and the persistent
// counting kernel, instantiated for every launch variant.
//
// The per-item algorithm is the paper's (arXiv 2412.16370, Section 4); the
// batching (work items, prefix sums, dynamic scheduling) is this library's.
#include "pospop_batch.cuh"

namespace pospop {

// Exclusive scan of the planning blocks' sums (one block), total into
// item_start[m], work counter reset.
__global__ void __launch_bounds__(kPlanThreads) plan_scan_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  __shared__ uint64_t carry;
  pdl_enter();
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

// item_start[a] = exclusive prefix sum of the per-array item counts.
__global__ void __launch_bounds__(kPlanThreads) plan_apply_kernel(PlanParams P) {
  __shared__ uint64_t red[32];
  pdl_enter();
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

#define POSPOP_BV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&batch_kernel<kSrcCsr, BS, MINB, D, H>), BS, MINB, D, H}

static const Variant kBatch[] = {POSPOP_FAMILY(POSPOP_BV)};

#define POSPOP_BV256(BS, MINB, D, H)                                                         \
  Variant{reinterpret_cast<const void *>(&batch_kernel<kSrcCsr, BS, MINB, D, H, true>), BS, \
          MINB, D, H}
static const Variant kBatch256[] = {POSPOP_FAMILY256(POSPOP_BV256)};

int batch_variant_count() { return (int)(sizeof(kBatch) / sizeof(kBatch[0])); }
const Variant &batch_variant(int i) { return kBatch[i]; }
int batch256_variant_count() { return (int)(sizeof(kBatch256) / sizeof(kBatch256[0])); }
const Variant &batch256_variant(int i) { return kBatch256[i]; }

const void *plan_items_fn() { return reinterpret_cast<const void *>(&plan_items_kernel<kSrcCsr>); }
const void *plan_scan_fn() { return reinterpret_cast<const void *>(&plan_scan_kernel); }
const void *plan_apply_fn() { return reinterpret_cast<const void *>(&plan_apply_kernel); }

}  // namespace pospop

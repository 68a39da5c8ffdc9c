// pospop_gather.cu -- counting several separate regions into one counter
// array (pospopcnt_gather).  Each region is its own word stream (its start
// fixes its phase), exactly as if each were counted alone into the same
// counters: the paper's add-into contract (Section 4, step 1 and its
// footnote) used for non-contiguous input.  Same planning and persistent
// counting templates as the CSR batch; the per-block counters meet in shared
// memory and reach global memory with one atomic per counter per block.
#include "pospop_batch.cuh"

namespace pospop {

#define POSPOP_GV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&batch_kernel<kSrcGather, BS, MINB, D, H>), BS, MINB, D, H}

static const Variant kGather[] = {POSPOP_FAMILY(POSPOP_GV)};

#define POSPOP_GV256(BS, MINB, D, H)                                                            \
  Variant{reinterpret_cast<const void *>(&batch_kernel<kSrcGather, BS, MINB, D, H, true>), BS, \
          MINB, D, H}
static const Variant kGather256[] = {POSPOP_FAMILY256(POSPOP_GV256)};

int gather_variant_count() { return (int)(sizeof(kGather) / sizeof(kGather[0])); }
const Variant &gather_variant(int i) { return kGather[i]; }
int gather256_variant_count() { return (int)(sizeof(kGather256) / sizeof(kGather256[0])); }
const Variant &gather256_variant(int i) { return kGather256[i]; }

const void *plan_items_gather_fn() {
  return reinterpret_cast<const void *>(&plan_items_kernel<kSrcGather>);
}

}  // namespace pospop

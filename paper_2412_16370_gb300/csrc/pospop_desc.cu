// pospop_desc.cu -- the batched counting kernel over per-array descriptors
// (pointer, length, w, output row), used by the serving loop to count
// requests of mixed width and size in one launch.  Same planning and
// counting templates as pospop_batch.cu.
#include "pospop_batch.cuh"

namespace pospop {

#define POSPOP_DV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&batch_kernel<kSrcDesc, BS, MINB, D, H>), BS, MINB, D, H}

static const Variant kDesc[] = {POSPOP_FAMILY(POSPOP_DV)};

int desc_variant_count() { return (int)(sizeof(kDesc) / sizeof(kDesc[0])); }
const Variant &desc_variant(int i) { return kDesc[i]; }

const void *plan_items_desc_fn() { return reinterpret_cast<const void *>(&plan_items_kernel<kSrcDesc>); }

}  // namespace pospop

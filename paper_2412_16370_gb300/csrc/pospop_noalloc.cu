// pospop_noalloc.cu -- pospopcnt_batch_noalloc: the batched count over CSR
// offsets for callers that cannot allocate device memory.
//
// pospopcnt_batch needs scratch memory for its work plan (per-array prefix
// sums of work items, the planning blocks' sums, a work counter and a status
// word) and takes it from a per-stream workspace that it grows with
// cudaMalloc whenever a batch has more arrays than before.  Some callers
// cannot let that happen: code that is recording a CUDA graph in a capture
// mode that rejects allocation, services that must not allocate once they
// are running (fixed memory footprint, no allocator stalls on the request
// path), and programs whose device memory is already handed out by another
// allocator.  This entry point takes the same arguments and launches the same
// planning and counting kernels, but keeps its scratch in a fixed array that
// is part of the library's own device image.
//
// The array (`g_noalloc_scratch` below) is a file-scope __device__ array:
// every GPU that loads the library holds it (about 513 KiB) until the
// process exits, and its size caps a call at kNoAllocMaxArrays arrays.  Host
// code cannot use the array's name as a device address, so the first call on
// each device, with that device current, looks the address up with
// cudaGetSymbolAddress and keeps it; make that first call before capturing
// any stream.  All calls share the one array, which keeps the last call's
// contents: the status word is cleared at the start of every call and the
// planning kernels rewrite everything else before it is read.  Calls that
// overlap on the GPU (on two streams at once, or from two host threads
// without ordering) race on the array and give wrong counts; order them.
#include <mutex>

#include "pospopcnt.h"
#include "pospop_runtime.h"

namespace pospop {
namespace {

constexpr size_t kNoAllocMaxArrays = 65535;
constexpr size_t kNoAllocBlocks = (kNoAllocMaxArrays + kPlanChunk - 1) / kPlanChunk;
// item_start (m + 1), planning block sums, work counter, status word.
constexpr size_t kItemStartBytes = 8 * (kNoAllocMaxArrays + 1);
constexpr size_t kBlockSumBytes = 8 * kNoAllocBlocks;
constexpr size_t kNoAllocScratchBytes = kItemStartBytes + kBlockSumBytes + 16;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (the current device).
int scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return POSPOP_ECUDA;
    }
    g_noalloc_ptr[device] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_ptr[device];
  return POSPOP_OK;
}

bool noalloc_valid_w(int w) {
  return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64;
}

bool noalloc_addressable(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

}  // namespace
}  // namespace pospop

using namespace pospop;

extern "C" int pospopcnt_batch_noalloc(int w, uint64_t *counts, const void *base,
                                       const uint64_t *offsets, size_t m, void *stream) {
  if (!noalloc_valid_w(w)) return POSPOP_EINVAL;
  if (m == 0) return POSPOP_OK;
  if (!counts || !base || !offsets) return POSPOP_EINVAL;
  if (m > kNoAllocMaxArrays) return POSPOP_ERANGE;
  int rc = POSPOP_OK;
  DevCtx *c = current_ctx(&rc);
  if (!c) return rc;
  if (!noalloc_addressable(counts, c->device) || !noalloc_addressable(base, c->device) ||
      !noalloc_addressable(offsets, c->device))
    return POSPOP_EPTR;
  unsigned char *scratch = nullptr;
  rc = scratch_address(c->device, &scratch);
  if (rc != POSPOP_OK) return rc;
  BatchTune bt;
  uint32_t regroup;
  {
    std::lock_guard<std::mutex> g(c->mu);
    bt = c->tune.batch[width_group(w)];
    regroup = c->tune.regroup;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t *item_start = reinterpret_cast<uint64_t *>(scratch);
  uint64_t *block_sum = reinterpret_cast<uint64_t *>(scratch + kItemStartBytes);
  unsigned long long *next =
      reinterpret_cast<unsigned long long *>(scratch + kItemStartBytes + kBlockSumBytes);
  int *status = reinterpret_cast<int *>(scratch + kItemStartBytes + kBlockSumBytes + 8);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }

  PlanParams pp;
  pp.gptrs = nullptr;
  pp.glens = nullptr;
  pp.offsets = offsets;
  pp.m = m;
  pp.base_addr = (uint64_t)base;
  pp.item_start = item_start;
  pp.block_sum = block_sum;
  pp.next = next;
  pp.status = status;
  pp.item_rows = bt.item_rows;
  pp.nblocks = (uint32_t)((m + kPlanChunk - 1) / kPlanChunk);
  void *pargs[] = {&pp};
  if (cudaLaunchKernel(plan_items_fn(), dim3(pp.nblocks), dim3(kPlanThreads), pargs, 0, s) !=
          cudaSuccess ||
      cudaLaunchKernel(plan_scan_fn(), dim3(1), dim3(kPlanThreads), pargs, 0, s) != cudaSuccess ||
      cudaLaunchKernel(plan_apply_fn(), dim3(pp.nblocks), dim3(kPlanThreads), pargs, 0, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }

  BatchParams bp;
  bp.gptrs = nullptr;
  bp.glens = nullptr;
  bp.base = static_cast<const uint8_t *>(base);
  bp.offsets = offsets;
  bp.m = m;
  bp.counts = reinterpret_cast<unsigned long long *>(counts);
  bp.w = w;
  bp.item_start = item_start;
  bp.next = next;
  bp.status = status;
  bp.item_rows = bt.item_rows;
  bp.grab = bt.grab;
  bp.regroup = regroup;
  const Variant &v = batch_variant(bt.variant);
  int cps = bt.ctas_per_sm < c->occ_batch[bt.variant] ? bt.ctas_per_sm : c->occ_batch[bt.variant];
  if (cps < 1) cps = 1;
  void *bargs[] = {&bp};
  if (cudaLaunchKernel(v.fn, dim3((unsigned)(c->sms * cps)), dim3(v.bs), bargs, 0, s) !=
      cudaSuccess) {
    cudaGetLastError();
    return POSPOP_ECUDA;
  }
  note_launches(4);
  return POSPOP_OK;
}

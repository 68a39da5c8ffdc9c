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
// code cannot use the array's name as a device address: when the library
// sets a device up (pospopcnt_init, or the first call of any entry point on
// that device), it looks the address up with cudaGetSymbolAddress, with that
// device current, and keeps it; make that first call before capturing any
// stream.  All calls share the one array, which keeps the last call's
// contents: the status word is cleared at the start of every call and the
// planning kernels rewrite everything else before it is read.  Calls that
// overlap on the GPU (on two streams at once, or from two host threads
// without ordering) race on the array and give wrong counts; order them.
#include "pospopcnt.h"
#include "pospop_runtime.h"

namespace pospop {
namespace {

constexpr size_t kNoAllocMaxArrays = 65535;
// item_start (m + 1), planning block sums, work counter, status word: the
// layout of a workspace for kNoAllocMaxArrays arrays.
constexpr size_t kNoAllocScratchBytes = scratch_bytes(kNoAllocMaxArrays);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

bool noalloc_valid_w(int w) {
  return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64;
}

}  // namespace

int noalloc_lookup(unsigned char **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    *out = nullptr;
    return POSPOP_ECUDA;
  }
  *out = static_cast<unsigned char *>(p);
  return POSPOP_OK;
}

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
  if (!c->noalloc_scratch) return POSPOP_ECUDA;
  // the same pointer rules as pospopcnt_batch (mapped host memory is given
  // to the kernels by its device address)
  const void *dc = nullptr, *db = nullptr, *doff = nullptr;
  if (!device_addressable(counts, c->device, &dc) || !device_addressable(base, c->device, &db) ||
      !device_addressable(offsets, c->device, &doff))
    return POSPOP_EPTR;
  TuneTable t;
  {
    std::lock_guard<std::mutex> g(c->mu);
    t = c->tune;
  }
  const Scratch scr = scratch_layout(c->noalloc_scratch, kNoAllocMaxArrays);
  return launch_batch_scratch(*c, t, w, (unsigned long long *)const_cast<void *>(dc), db,
                              static_cast<const uint64_t *>(doff), m, scr,
                              static_cast<cudaStream_t>(stream));
}

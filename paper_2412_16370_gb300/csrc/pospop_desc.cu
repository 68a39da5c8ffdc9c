// pospop_desc.cu -- the serving loop's counting kernel (and its add-into
// form behind pospopcnt_multi): one launch counts up to kServeMax requests
// of mixed width and size, passed by value in the kernel's parameter block
// (a __grid_constant__ struct, read in place through the constant cache: no
// upload copy before the launch; about 14 KiB, or about 1 KiB in the form
// for at most kServeSmall requests).
//
// A launch counts work items [item0, item0 + its items here) of each
// request, so one request's items may be spread over several launches; its
// slot's completion counter counts them all.  Work items (req.rows rows of
// 512 B of one request, as in the batched
// count: either a contiguous run of rows, or with `strided` every K-th row
// of a request of K items, so that warps on neighbouring items read
// neighbouring rows as the single-array kernel's warps do) are dealt to
// warps round-robin; each is counted with the paper's
// per-thread algorithm (Section 4) and folded into its request slot's
// counters.  The warp that finishes a request's last work item reads and
// clears its counters, resets the slot's completion counter, publishes the
// counts to mapped pinned host memory and then raises the request's flag,
// so a request completes without waiting for the rest of the launch and the
// slot's device state is clean for the next launch (no memset between
// launches).  Fences: device scope before each completion count (this
// warp's counter atomics first), device scope before the read-and-clear,
// system scope before the flag.
#include "pospop_batch.cuh"

namespace pospop {

// Largest k in [0, n) with item_start[k] <= i (item_start[0] = 0 <= i <
// item_start[n]), 32-way warp search over the parameter block.
__device__ __forceinline__ uint32_t find_request(const uint64_t *item_start, uint32_t n,
                                                 uint64_t i, unsigned lane) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t span = hi - lo;
    const uint32_t idx = lo + (uint32_t)((uint64_t)span * (lane + 1) / 33);
    const unsigned b = __ballot_sync(kFull, item_start[idx] <= i);
    const int c = __popc(b);
    const uint32_t nlo = c > 0 ? lo + (uint32_t)((uint64_t)span * c / 33) : lo;
    const uint32_t nhi = c < 32 ? lo + (uint32_t)((uint64_t)span * (c + 1) / 33) : hi;
    lo = nlo;
    hi = nhi > lo ? nhi : lo + 1;
  }
  return lo;
}

// ADD: the add-into form of pospopcnt_multi: every work item's counts are
// added straight into its count's own counters (req.out), with no request
// slots and no completion tracking; it waits for the previous kernel on the
// stream (programmatic dependent launch) like the other counting kernels.
template <int BS, int MINB, int DEPTH, int HINT, bool ADD = false, int N = kServeMax>
__global__ void __launch_bounds__(BS, MINB)
    serve_kernel(const __grid_constant__ ServeParamsT<N> P) {
  if (ADD) pdl_enter();
  constexpr unsigned WPB = BS / 32;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t NW = (uint64_t)gridDim.x * WPB;
  const Xpose xk = make_xpose(lane);
  for (uint64_t i = (uint64_t)blockIdx.x * WPB + (threadIdx.x >> 5); i < P.total; i += NW) {
    const uint32_t k = find_request(P.item_start, P.n, i, lane);
    const ServeReq &rq = P.req[k];
    const uint64_t s0 = (uint64_t)rq.ptr, e0 = s0 + rq.nbytes;
    Span s;
    const uint64_t A = s0 & ~15ull;
    s.A = reinterpret_cast<const uint8_t *>(A);
    s.head = (uint32_t)(s0 - A);
    s.G = (((e0 + 15u) & ~15ull) - A) >> 4;
    s.tail = (uint32_t)(e0 - (A + 16u * (s.G - 1)));
    const int w = rq.w;
    const uint32_t rot = (8u * s.head) & (uint32_t)(w - 1);
    const uint64_t R = span_rows(s);
    const uint64_t kk = rq.item0 + (i - P.item_start[k]);   // the item's index within its request
    uint64_t r0, stride, nrows;
    if (P.strided) {
      // rows kk, kk + K, ...: at most ceil(R / K) <= rq.rows of them
      // (32-bit: the host keeps strided requests below 2^32 rows, and a
      // 64-bit division's call would spill the CSA state)
      const uint32_t K = rq.items, k32 = (uint32_t)kk, R32 = (uint32_t)R;
      r0 = kk;
      stride = K;
      nrows = R32 > k32 ? (R32 - k32 - 1) / K + 1 : 0;
    } else {
      r0 = kk * rq.rows;
      stride = 1;
      nrows = ((r0 + rq.rows < R) ? r0 + rq.rows : R) - r0;
    }
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    count_rows<DEPTH, HINT>(s, r0, stride, nrows, lane, xk, cnt, PlainLoader<HINT>{});
    if (ADD) {
      unsigned long long *dst = rq.out;
      fold_counts(cnt, w, rot, lane, [&](uint32_t j, unsigned long long v) {
        if (v) atomicAdd(dst + j, v);
      });
      continue;
    }
    const uint32_t slot = rq.slot;
    unsigned long long *out = P.counts + 64ull * slot;
    fold_counts(cnt, w, rot, lane, [&](uint32_t j, unsigned long long v) {
      if (v) atomicAdd(out + j, v);
    });
    // completion of request k
    __threadfence();
    unsigned last = 0;
    if (lane == 0) last = atomicAdd(P.done + slot, 1u) + 1u == rq.items ? 1u : 0u;
    last = __shfl_sync(kFull, last, 0);
    if (last) {
      __threadfence();
      unsigned long long *res = P.host_res + 64ull * slot;
      for (int j = (int)lane; j < w; j += 32) res[j] = atomicExch(out + j, 0ull);
      if (lane == 0) atomicExch(P.done + slot, 0u);
      __threadfence_system();
      __syncwarp();
      if (lane == 0) {
        __threadfence_system();
        *reinterpret_cast<volatile unsigned int *>(P.flags + slot) = rq.seq;
        __threadfence_system();
      }
    }
  }
}

#define POSPOP_SERV(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&serve_kernel<BS, MINB, D, H>), BS, MINB, D, H}
#define POSPOP_SERV_S(BS, MINB, D, H)                                                        \
  Variant{reinterpret_cast<const void *>(&serve_kernel<BS, MINB, D, H, false, kServeSmall>), \
          BS, MINB, D, H}

static const Variant kServe[] = {POSPOP_FAMILY(POSPOP_SERV)};
static const Variant kServeSm[] = {POSPOP_FAMILY(POSPOP_SERV_S)};

int serve_variant_count() { return (int)(sizeof(kServe) / sizeof(kServe[0])); }
const Variant &serve_variant(int i) { return kServe[i]; }
const Variant &serve_small_variant(int i) { return kServeSm[i]; }

#define POSPOP_MULTI(BS, MINB, D, H) \
  Variant{reinterpret_cast<const void *>(&serve_kernel<BS, MINB, D, H, true>), BS, MINB, D, H}
#define POSPOP_MULTI_S(BS, MINB, D, H)                                                      \
  Variant{reinterpret_cast<const void *>(&serve_kernel<BS, MINB, D, H, true, kServeSmall>), \
          BS, MINB, D, H}

static const Variant kMulti[] = {POSPOP_FAMILY(POSPOP_MULTI)};
static const Variant kMultiSm[] = {POSPOP_FAMILY(POSPOP_MULTI_S)};

int multi_variant_count() { return (int)(sizeof(kMulti) / sizeof(kMulti[0])); }
const Variant &multi_variant(int i) { return kMulti[i]; }
const Variant &multi_small_variant(int i) { return kMultiSm[i]; }

}  // namespace pospop

// pospop_device.cuh -- device building blocks of the sm_103a positional
// population count (arXiv 2412.16370, Sections 3-4), shared by the
// single-array, batched and serving kernels.
//
// Data layout.  The input byte stream is cut into 16-byte granules aligned
// to 16 bytes (the first granule starts at the start address rounded down).
// One granule is four 32-bit lanes: lane r holds granule bit positions
// 32r .. 32r+31, and granule bit position k = 8 * (byte in granule) + bit.
// A "row" is 32 consecutive granules (512 bytes); lane l of a warp always
// handles granule l of a row, so every warp-wide load is one coalesced
// 512-byte row.  Because 16-byte granules are aligned and w divides 128,
// granule bit position k always belongs to counter (k - 8*head) mod w, where
// head is the start's offset past the 16-byte boundary.
//
// Per thread, the granules of the rows a thread visits are reduced in
// registers with the paper's carry-save-adder (CSA) networks: CSA_15 for the
// first 15 vectors (Section 4.2, 11 full adders), then CSA_16+4 for every
// further 16 (15 full adders), each full adder being two lop3 instructions
// (Section 3.1.1, Eq. 3: parity 0x96 for the sum, majority 0xe8 for the
// carry).  The a16 bit vector skimmed off every 16 vectors (Section 4.3,
// Eq. 4) is counted with a 32x32 bit transpose across the warp followed by
// one popcount per lane, which yields the warp-wide count of one bit
// position per lane; the final (a8, a4, a2, a1) vectors are counted the same
// way with weights 8, 4, 2, 1 (Section 4.5).  Counters are u32 per lane and
// position; the host bounds the rows per warp so they cannot overflow (the
// role of Eq. 5, Section 4.4).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pospop {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGranule = 16;               // bytes per granule (one uint4 per lane)
constexpr int kRowBytes = 32 * kGranule;   // 512 bytes per warp row

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may be scheduled while the kernel before it on the stream is
// still running.  griddepcontrol.wait blocks until that kernel has completed
// and its memory operations are visible, so every kernel below runs it before
// touching global memory: stream order is kept exactly, and only the launch
// itself overlaps the previous kernel.  griddepcontrol.launch_dependents then
// lets the next such kernel be scheduled.  Without the launch attribute both
// instructions have no effect.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Bit-parallel full adder (Section 3.1.1, Eq. 3): one lop3 per output.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lop3_parity(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t lop3_majority(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0xe8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

struct V4 {
  uint32_t x[4];
};

__device__ __forceinline__ V4 v4_zero() { return V4{{0u, 0u, 0u, 0u}}; }

// (carry, sum) = FA(a, b, c) on all 128 bits of a granule.
__device__ __forceinline__ void fa(V4 &sum, V4 &carry, const V4 &a, const V4 &b, const V4 &c) {
  V4 s, k;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    s.x[r] = lop3_parity(a.x[r], b.x[r], c.x[r]);
    k.x[r] = lop3_majority(a.x[r], b.x[r], c.x[r]);
  }
  sum = s;
  carry = k;
}

// Half adder, used only to merge a16 vectors into the deeper a16 plane.
__device__ __forceinline__ void ha(V4 &sum, V4 &carry, const V4 &a, const V4 &b) {
  V4 s, k;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    s.x[r] = a.x[r] ^ b.x[r];
    k.x[r] = a.x[r] & b.x[r];
  }
  sum = s;
  carry = k;
}

// Bit-sliced per-thread accumulator: weights 1, 2, 4, 8 (and 16 when the
// flush depth is 32 vectors).
struct Planes {
  V4 a1, a2, a4, a8, a16;
};

// CSA_15 (Section 4.2): 15 vectors of weight 1 -> (a8, a4, a2, a1) with 11
// full adders and a critical path of 5.
__device__ __forceinline__ void csa15(Planes &p, const V4 *v) {
  V4 s0, s1, s2, s3, s4, c0, c1, c2, c3, c4;
  fa(s0, c0, v[0], v[1], v[2]);
  fa(s1, c1, v[3], v[4], v[5]);
  fa(s2, c2, v[6], v[7], v[8]);
  fa(s3, c3, v[9], v[10], v[11]);
  fa(s4, c4, v[12], v[13], v[14]);
  V4 t0, d0, d1;
  fa(t0, d0, s0, s1, s2);
  fa(p.a1, d1, t0, s3, s4);          // weight 1 done
  V4 u0, u1, e0, e1, e2;
  fa(u0, e0, c0, c1, c2);
  fa(u1, e1, c3, c4, d0);
  fa(p.a2, e2, u0, u1, d1);          // weight 2 done
  fa(p.a4, p.a8, e0, e1, e2);        // weights 4 and 8
}

// CSA_16+4 (Section 4.2): 16 vectors of weight 1 plus (a8, a4, a2, a1) ->
// (a16, a8, a4, a2, a1) with 15 full adders.  Returns a16.
__device__ __forceinline__ V4 csa16(Planes &p, const V4 *v) {
  V4 s0, s1, s2, s3, s4, c0, c1, c2, c3, c4;
  fa(s0, c0, p.a1, v[0], v[1]);
  fa(s1, c1, v[2], v[3], v[4]);
  fa(s2, c2, v[5], v[6], v[7]);
  fa(s3, c3, v[8], v[9], v[10]);
  fa(s4, c4, v[11], v[12], v[13]);
  V4 t0, t1, d0, d1, d2;
  fa(t0, d0, s0, s1, s2);
  fa(t1, d1, s3, s4, v[14]);
  fa(p.a1, d2, t0, t1, v[15]);       // weight 1: 8 full adders
  V4 u0, u1, u2, e0, e1, e2, e3;
  fa(u0, e0, p.a2, c0, c1);
  fa(u1, e1, c2, c3, c4);
  fa(u2, e2, d0, d1, d2);
  fa(p.a2, e3, u0, u1, u2);          // weight 2: 4 full adders
  V4 x0, f0, f1;
  fa(x0, f0, p.a4, e0, e1);
  fa(p.a4, f1, x0, e2, e3);          // weight 4: 2 full adders
  V4 a16;
  fa(p.a8, a16, p.a8, f0, f1);       // weight 8: 1 full adder
  return a16;
}

// ---------------------------------------------------------------------------
// Warp-wide 32x32 bit transpose + popcount.
//
// Lane t holds row t (a 32-bit register).  Five exchange stages (distance
// 16, 8, 4, 2, 1) each swap bit j of the row index with bit j of the column
// index; afterwards lane l holds column l, i.e. bit l of every lane's
// register, and its popcount is the warp-wide count of bit position l.
// Per stage: one funnel-shift rotate, one shuffle, one lop3 select.
// ---------------------------------------------------------------------------
struct Xpose {
  uint32_t amt[5];
  uint32_t keep[5];
};

__device__ __forceinline__ Xpose make_xpose(unsigned lane) {
  const uint32_t low[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
  Xpose k;
#pragma unroll
  for (int s = 0; s < 5; s++) {
    const unsigned j = 16u >> s;
    const bool lower = (lane & j) == 0;
    k.amt[s] = lower ? j : 32u - j;     // lower lanes send rotr(x, j), upper lanes rotl(x, j)
    k.keep[s] = lower ? low[s] : ~low[s];
  }
  return k;
}

__device__ __forceinline__ uint32_t xpose_popc(uint32_t x, const Xpose &k) {
#pragma unroll
  for (int s = 0; s < 5; s++) {
    const unsigned j = 16u >> s;
    const uint32_t send = __funnelshift_r(x, x, k.amt[s]);
    const uint32_t y = __shfl_xor_sync(kFull, send, j);
    x = (x & k.keep[s]) | (y & ~k.keep[s]);
  }
  return (uint32_t)__popc(x);
}

// cnt[r] += weight * (warp-wide count of granule position 32r + lane in v).
template <int SHIFT>
__device__ __forceinline__ void flush_plane(uint32_t cnt[4], const V4 &v, const Xpose &k) {
#pragma unroll
  for (int r = 0; r < 4; r++) cnt[r] += xpose_popc(v.x[r], k) << SHIFT;
}

// Flush for w = 256, where a word spans two granules: granule g's bits
// belong to word half g mod 2, and g mod 2 is the lane's parity (rows start
// at even granules), so even and odd lanes are transposed and counted apart.
template <int SHIFT, bool PAR2>
__device__ __forceinline__ void flush_par(uint32_t cnt[4], uint32_t cnt_odd[4], const V4 &v,
                                          const Xpose &k, unsigned lane) {
  if (PAR2) {
    const uint32_t odd = 0u - (lane & 1u);
#pragma unroll
    for (int r = 0; r < 4; r++) {
      cnt[r] += xpose_popc(v.x[r] & ~odd, k) << SHIFT;
      cnt_odd[r] += xpose_popc(v.x[r] & odd, k) << SHIFT;
    }
  } else {
    flush_plane<SHIFT>(cnt, v, k);
  }
}

// ---------------------------------------------------------------------------
// Loads.
// ---------------------------------------------------------------------------
// HINT 0: ld.global.nc with L1 no-allocate; HINT 1: additionally asks L2 to
// fetch 256-byte sectors (streaming prefetch).
template <int HINT>
__device__ __forceinline__ V4 ldg_granule(const uint8_t *p) {
  V4 v;
  if (HINT == 1) {
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x[0]), "=r"(v.x[1]), "=r"(v.x[2]), "=r"(v.x[3])
        : "l"(p));
  } else {
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x[0]), "=r"(v.x[1]), "=r"(v.x[2]), "=r"(v.x[3])
        : "l"(p));
  }
  return v;
}

// One array (or a piece of one) in granule coordinates.
struct Span {
  const uint8_t *A;   // 16-byte aligned address of granule 0
  uint64_t G;         // granules (>= 1)
  uint32_t head;      // bytes of granule 0 before the first counted byte (0..15)
  uint32_t tail;      // counted bytes of granule G-1 (1..16)
};

__host__ __device__ __forceinline__ uint64_t span_rows(const Span &s) { return (s.G + 31) >> 5; }

// Bytes [lo, hi) of the granule at p, the rest zero.  Not inlined: a span
// has at most two partial granules, and keeping this loop out of the
// dozens of unrolled load sites of count_rows keeps the kernels' code small
// enough for the instruction cache when warps work on many short arrays at
// once (measured on GB300: 100000 gathered regions counted 15% faster).
static __device__ __noinline__ V4 load_partial_granule(const uint8_t *p, uint32_t lo, uint32_t hi) {
  V4 v = v4_zero();
  for (uint32_t b = lo; b < hi; b++) {
    const uint32_t byte = __ldg(p + b);
    v.x[b >> 2] |= byte << (8u * (b & 3u));
  }
  return v;
}

// Granule g with everything outside the span zeroed.  Bytes outside
// [start, end) are never read: the partial first and last granules are read
// byte by byte.
template <int HINT>
__device__ __forceinline__ V4 load_granule_masked(const Span &s, uint64_t g) {
  if (g >= s.G) return v4_zero();
  const uint32_t lo = (g == 0) ? s.head : 0u;
  const uint32_t hi = (g == s.G - 1) ? s.tail : 16u;
  const uint8_t *p = s.A + g * kGranule;
  if (lo == 0u && hi == 16u) return ldg_granule<HINT>(p);
  return load_partial_granule(p, lo, hi);
}

// ---------------------------------------------------------------------------
// Loader policies.  count_rows fetches granules through a loader: `group16`
// for a CSA group of 16 rows known to lie wholly inside the span, `edge` for
// any granule (bytes outside the span read as zero).  PlainLoader is the
// plain count; SelectLoader (below) also applies a word-selection bitmap.
// ---------------------------------------------------------------------------
template <int HINT>
struct PlainLoader {
  __device__ __forceinline__ V4 edge(const Span &s, uint64_t g) const {
    return load_granule_masked<HINT>(s, g);
  }
  // 16 interior granules: row k at ptr + k * pstep (granule g + k * gstride).
  __device__ __forceinline__ void group16(V4 (&v)[16], const uint8_t *ptr, uint64_t pstep, uint64_t,
                                          uint64_t) const {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = ldg_granule<HINT>(ptr + (uint64_t)k * pstep);
  }
};

// Word selection (the WHERE bitmap of a GROUP BY count, Section 1): bit i of
// the bitmap (least significant bit of byte i/8 first) selects word i of the
// span, whose start is a multiple of the word size W = 2^WLOG bytes.
struct Selection {
  const uint8_t *bits;   // bitmap, 4-byte aligned, ceil(nbits / 32) readable 32-bit words
  uint64_t nbits;        // words in the span (selection bits that count)
  uint64_t nbytes;       // readable bytes of the bitmap (4 * ceil(nbits / 32))
  uint32_t h;            // words before the start in granule 0 (span head / W)
};

// 32 bitmap bits starting at bit 32q (bits past the readable bytes read as 0).
__device__ __forceinline__ uint32_t sel_word(const Selection &m, uint64_t q) {
  const uint64_t b0 = 4 * q;
  if (b0 + 4 <= m.nbytes) return __ldg(reinterpret_cast<const uint32_t *>(m.bits) + q);
  uint32_t v = 0;
  for (uint64_t b = b0; b < m.nbytes && b < b0 + 4; b++) v |= (uint32_t)__ldg(m.bits + b) << (8 * (b - b0));
  return v;
}

// Selection bits of granule g: bit t (t < 16 / W) selects the word that
// occupies bytes [t W, (t + 1) W) of the granule.
template <int WLOG>
__device__ __forceinline__ uint32_t granule_selection(const Selection &m, uint64_t g) {
  constexpr uint32_t CNT = 16u >> WLOG;
  constexpr uint32_t ALL = (1u << CNT) - 1u;
  const uint64_t gb = g * CNT;
  uint32_t bits;
  uint64_t lo;
  uint32_t lead;   // selection slots before the start (granule 0 only)
  if (gb >= m.h) {
    lo = gb - m.h;
    lead = 0;
  } else {
    lo = 0;
    lead = (uint32_t)(m.h - gb);
  }
  const uint64_t q = lo >> 5;
  const uint32_t sh = (uint32_t)lo & 31u;
  const uint32_t w0 = sel_word(m, q);
  const uint32_t w1 = (sh + CNT > 32u) ? sel_word(m, q + 1) : 0u;
  bits = __funnelshift_r(w0, w1, sh) << lead;
  if (lo + CNT > m.nbits + lead) {   // selection bits past the last word do not count
    const uint64_t keep = (m.nbits > lo ? m.nbits - lo : 0) + lead;
    if (keep < 32) bits &= (1u << (uint32_t)keep) - 1u;
  }
  return bits & ALL;
}

// Byte mask of one 32-bit lane from its selection bits.  prmt with the
// sign-replicate selector copies bit 7 of a chosen byte over the whole byte,
// so the selection bits are first moved (one multiply, no carries since the
// shifted copies do not overlap) to bit 7 of the bytes they cover.
template <int WLOG>
__device__ __forceinline__ uint32_t lane_mask(uint32_t bits, int r) {
  uint32_t e;
  if (WLOG == 0) {          // w = 8: bit k of the nibble -> byte k
    const uint32_t t = ((bits >> (4 * r)) & 0xfu) * 0x10204080u;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(e) : "r"(t));
  } else if (WLOG == 1) {   // w = 16: bit k of the pair -> 16-bit half k
    const uint32_t t = ((bits >> (2 * r)) & 0x3u) * 0x40008000u;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(e) : "r"(t));
  } else if (WLOG == 2) {   // w = 32: one bit per lane, sign-extended by bfe
    asm("bfe.s32 %0, %1, %2, 1;" : "=r"(e) : "r"(bits), "r"(r));
  } else {                  // w = 64: one bit per two lanes
    asm("bfe.s32 %0, %1, %2, 1;" : "=r"(e) : "r"(bits), "r"(r >> 1));
  }
  return e;
}

template <int WLOG>
__device__ __forceinline__ void apply_selection(V4 &v, uint32_t bits) {
#pragma unroll
  for (int r = 0; r < 4; r++) v.x[r] &= lane_mask<WLOG>(bits, r);
}

template <int HINT, int WLOG>
struct SelectLoader {
  Selection m;
  // 16 interior granules g + k * gstride (not granule 0, not in the last
  // row): every selection window lies inside the span, so none needs
  // clipping.  Consecutive rows' windows lie stride * CNT bitmap words apart
  // at the same bit offset (gstride * CNT is a multiple of 32), so the window
  // address is one add per row and the offset and the straddle test are
  // shared by the group.  The second bitmap word is read only where a window
  // straddles into it (a predicated load); it then holds bits of the span's
  // words, so it lies inside the bitmap.  With a 16-byte-aligned start no
  // window straddles.
  __device__ __forceinline__ void group16(V4 (&v)[16], const uint8_t *ptr, uint64_t pstep,
                                          uint64_t g, uint64_t gstride) const {
    constexpr uint32_t CNT = 16u >> WLOG;
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = ldg_granule<HINT>(ptr + (uint64_t)k * pstep);
    const uint64_t lo = g * CNT - m.h;
    const uint32_t sh = (uint32_t)lo & 31u;
    const bool straddle = sh + CNT > 32u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(m.bits) + (lo >> 5);
    const uint64_t wstep = (gstride >> 5) * CNT;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint32_t *wk = w + (uint64_t)k * wstep;
      const uint32_t w0 = __ldg(wk);
      const uint32_t w1 = straddle ? __ldg(wk + 1) : 0u;
      apply_selection<WLOG>(v[k], __funnelshift_r(w0, w1, sh));
    }
  }
  __device__ __forceinline__ V4 edge(const Span &s, uint64_t g) const {
    V4 v = load_granule_masked<HINT>(s, g);
    if (g < s.G) apply_selection<WLOG>(v, granule_selection<WLOG>(m, g));
    return v;
  }
};

// ---------------------------------------------------------------------------
// The per-thread algorithm (Section 4, steps 2-7) over a sequence of rows
// row0, row0 + stride, ..., nrows of them.  Lane `lane` handles granule
// 32 * row + lane of each row.  Adds the warp-wide counts of granule bit
// positions 32r + lane (r = 0..3) into cnt[r].  Warp-uniform control flow.
// ---------------------------------------------------------------------------
template <int DEPTH, int HINT, class Loader, bool PAR2 = false>
__device__ __forceinline__ void count_rows(const Span &s, uint64_t row0, uint64_t stride,
                                           uint64_t nrows, unsigned lane, const Xpose &xk,
                                           uint32_t cnt[4], const Loader &ld,
                                           uint32_t *cnt_odd = nullptr) {
  if (nrows == 0) return;
  const uint64_t R = span_rows(s);
  const uint64_t gstride = stride * 32u;          // granules between consecutive rows
  uint64_t g = row0 * 32u + lane;                 // this lane's granule in the current row

  if (nrows <= 3) {
    // Short sequence (Section 4.6): too few vectors for a CSA network to pay;
    // count every vector directly.
    for (uint64_t i = 0; i < nrows; i++, g += gstride) {
      const V4 v = ld.edge(s, g);
      flush_par<0, PAR2>(cnt, cnt_odd, v, xk, lane);
    }
    return;
  }

  Planes p;
  {
    // Head (Section 4.1) and initial CSA_15 reduction (Section 4.2).  The
    // masked loader zeroes bytes before the start and after the end.
    V4 v[15];
#pragma unroll
    for (int i = 0; i < 15; i++)
      v[i] = ((uint64_t)i < nrows) ? ld.edge(s, g + (uint64_t)i * gstride) : v4_zero();
    csa15(p, v);
  }
  p.a16 = v4_zero();
  uint64_t i = 15;
  g += 15u * gstride;

  // Main loop (Section 4, step 5): 16 vectors per CSA_16+4, a16 skimmed off
  // and counted.  Groups whose rows are all interior (not the first row,
  // not the last row of the span) load without masking.
  const uint8_t *ptr = s.A + g * kGranule;
  const uint64_t pstep = gstride * kGranule;
  if (DEPTH == 32) {
    for (; i + 32 <= nrows; i += 32, g += 32u * gstride, ptr += 32u * pstep) {
      const uint64_t first_row = row0 + i * stride, last_row = row0 + (i + 31) * stride;
      const bool interior = first_row >= 1 && last_row + 1 < R;
      V4 x, y;
      {
        V4 v[16];
        if (interior) {
          ld.group16(v, ptr, pstep, g, gstride);
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++) v[k] = ld.edge(s, g + (uint64_t)k * gstride);
        }
        x = csa16(p, v);
      }
      {
        V4 v[16];
        if (interior) {
          ld.group16(v, ptr + 16u * pstep, pstep, g + 16u * gstride, gstride);
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++) v[k] = ld.edge(s, g + (uint64_t)(16 + k) * gstride);
        }
        y = csa16(p, v);
      }
      V4 a32;
      fa(p.a16, a32, p.a16, x, y);
      flush_par<5, PAR2>(cnt, cnt_odd, a32, xk, lane);
    }
  }
  for (; i < nrows; i += 16, g += 16u * gstride, ptr += 16u * pstep) {
    const uint64_t first_row = row0 + i * stride;
    const bool full = i + 16 <= nrows;
    const bool interior = full && first_row >= 1 && row0 + (i + 15) * stride + 1 < R;
    V4 v[16];
    if (interior) {
      ld.group16(v, ptr, pstep, g, gstride);
    } else {
      // Tail (Section 4.6): rows past the sequence and bytes past the end are zero.
#pragma unroll
      for (int k = 0; k < 16; k++)
        v[k] = (i + (uint64_t)k < nrows) ? ld.edge(s, g + (uint64_t)k * gstride) : v4_zero();
    }
    const V4 a16 = csa16(p, v);
    if (DEPTH == 32) {
      V4 a32;
      ha(p.a16, a32, p.a16, a16);
      flush_par<5, PAR2>(cnt, cnt_odd, a32, xk, lane);
    } else {
      flush_par<4, PAR2>(cnt, cnt_odd, a16, xk, lane);
    }
  }

  // Final accumulation (Section 4.5): the carried planes with weights 8, 4, 2, 1.
  if (DEPTH == 32) flush_par<4, PAR2>(cnt, cnt_odd, p.a16, xk, lane);
  flush_par<3, PAR2>(cnt, cnt_odd, p.a8, xk, lane);
  flush_par<2, PAR2>(cnt, cnt_odd, p.a4, xk, lane);
  flush_par<1, PAR2>(cnt, cnt_odd, p.a2, xk, lane);
  flush_par<0, PAR2>(cnt, cnt_odd, p.a1, xk, lane);
}

// w = 256: even lanes hold word bits 0..127 of their granule's phase, odd
// lanes bits 128..255.
template <typename Emit>
__device__ __forceinline__ void fold_counts_256(const uint32_t cnt[4], const uint32_t cnt_odd[4],
                                                uint32_t rot, unsigned lane, Emit emit) {
#pragma unroll
  for (int r = 0; r < 4; r++) {
    emit((32u * r + lane - rot) & 255u, (unsigned long long)cnt[r]);
    emit((128u + 32u * r + lane - rot) & 255u, (unsigned long long)cnt_odd[r]);
  }
}

// ---------------------------------------------------------------------------
// Per-lane bit regroup for w = 8 (the Future Work section's regrouping: each
// byte collects the bits of one place value, then a per-byte popcount).
// Eight bytes form an 8x8 bit matrix (row b = byte b); after the transpose
// byte j holds bit j of all eight bytes, so its popcount is the number of
// those bytes with bit j set.  A lane keeps its class counts as bytes
// (classes 0..3 in acc_lo, 4..7 in acc_hi; at most 16 per granule, so up to
// 15 granules fit a byte); the warp's sums come from redux.sync.  Used as an
// alternative to the transpose flush for short sequences (at most 3 rows).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
  uint64_t t;
  t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

// Popcount of each byte of v, in place.
__device__ __forceinline__ uint32_t popc_bytes(uint32_t v) {
  v = v - ((v >> 1) & 0x55555555u);
  v = (v & 0x33333333u) + ((v >> 2) & 0x33333333u);
  return (v + (v >> 4)) & 0x0F0F0F0Fu;
}

__device__ __forceinline__ void regroup_add_w8(const V4 &v, uint32_t &acc_lo, uint32_t &acc_hi) {
  const uint64_t a = transpose8x8(((uint64_t)v.x[1] << 32) | v.x[0]);
  const uint64_t b = transpose8x8(((uint64_t)v.x[3] << 32) | v.x[2]);
  acc_lo += popc_bytes((uint32_t)a) + popc_bytes((uint32_t)b);
  acc_hi += popc_bytes((uint32_t)(a >> 32)) + popc_bytes((uint32_t)(b >> 32));
}

// Class counts (w = 8) of a short row sequence (nrows <= 3), per lane.
template <class Loader>
__device__ __forceinline__ void regroup_rows_w8(const Span &s, uint64_t row0, uint64_t stride,
                                                uint64_t nrows, unsigned lane, const Loader &ld,
                                                uint32_t &acc_lo, uint32_t &acc_hi) {
  uint64_t g = row0 * 32u + lane;
  for (uint64_t i = 0; i < nrows; i++, g += stride * 32u) regroup_add_w8(ld.edge(s, g), acc_lo, acc_hi);
}

// Warp sums of the eight classes (fields widened to 16 bits: at most
// 48 * 32 per class), emitted by lane 0.  For w = 8 the phase rotation is 0.
template <typename Emit>
__device__ __forceinline__ void regroup_emit_w8(uint32_t acc_lo, uint32_t acc_hi, unsigned lane,
                                                Emit emit) {
  const uint32_t s02 = __reduce_add_sync(kFull, acc_lo & 0x00ff00ffu);
  const uint32_t s13 = __reduce_add_sync(kFull, (acc_lo >> 8) & 0x00ff00ffu);
  const uint32_t s46 = __reduce_add_sync(kFull, acc_hi & 0x00ff00ffu);
  const uint32_t s57 = __reduce_add_sync(kFull, (acc_hi >> 8) & 0x00ff00ffu);
  if (lane == 0) {
    emit(0u, (unsigned long long)(s02 & 0xffffu));
    emit(1u, (unsigned long long)(s13 & 0xffffu));
    emit(2u, (unsigned long long)(s02 >> 16));
    emit(3u, (unsigned long long)(s13 >> 16));
    emit(4u, (unsigned long long)(s46 & 0xffffu));
    emit(5u, (unsigned long long)(s57 & 0xffffu));
    emit(6u, (unsigned long long)(s46 >> 16));
    emit(7u, (unsigned long long)(s57 >> 16));
  }
}

// ---------------------------------------------------------------------------
// Fold (f_w, Section 4.4) with the phase rotation for unaligned starts: the
// lane's counts of granule positions 32r + lane become counter
// (32r + lane - rot) mod w.  For w <= 32 all four lanes r share one counter,
// and lanes l, l + w, l + 2w, ... are summed with shuffles first.
// emit(j, value) is called by the lanes that own a finished counter.
// ---------------------------------------------------------------------------
template <typename Emit>
__device__ __forceinline__ void fold_counts(const uint32_t cnt[4], int w, uint32_t rot,
                                            unsigned lane, Emit emit) {
  if (w == 128) {            // a granule is one word phase class: no folding
#pragma unroll
    for (int r = 0; r < 4; r++) emit((32u * r + lane - rot) & 127u, (unsigned long long)cnt[r]);
  } else if (w == 64) {
    const unsigned long long v0 = (unsigned long long)cnt[0] + cnt[2];
    const unsigned long long v1 = (unsigned long long)cnt[1] + cnt[3];
    emit((lane - rot) & 63u, v0);
    emit((lane + 32u - rot) & 63u, v1);
  } else {
    unsigned long long v = (unsigned long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
    for (int off = 16; off >= w; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    if ((int)lane < w) emit((lane - rot) & (uint32_t)(w - 1), v);
  }
}

}  // namespace pospop

// synth.cu -- device twin of the seeded input generator (synth.py); see
// include/pospop_synth.h.  Generates inputs only; no counting here.
#include <cuda_runtime.h>

#include <cstdint>

#include "pospop_synth.h"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1u) * kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum Kind { kRandom = 0, kBernoulli = 1, kOneHot = 2, kFill = 3 };

struct Args {
  uint8_t *dst;
  uint64_t nbytes;
  uint64_t seed;
  uint64_t start;
  uint64_t threshold;
  uint32_t th[8];
  int nth;
  int kind;
  uint8_t value;
};

__device__ __forceinline__ uint8_t make_byte(const Args &a, uint64_t k) {
  switch (a.kind) {
    case kRandom:
      return (uint8_t)(splitmix64(a.seed, k >> 3) >> (8u * (k & 7u)));
    case kBernoulli: {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 8; b++)
        v |= (uint32_t)((splitmix64(a.seed, 8u * k + b) >> 32) < a.threshold) << b;
      return (uint8_t)v;
    }
    case kOneHot: {
      const uint32_t u = (uint32_t)(splitmix64(a.seed, k) >> 32);
      int c = 0;
      for (int t = 0; t < a.nth; t++) c += (u >= a.th[t]) ? 1 : 0;
      return (uint8_t)(1u << c);
    }
    default:
      return a.value;
  }
}

// Each thread writes 16 consecutive output bytes; aligned full chunks are
// stored with one 16-byte store.
__global__ void synth_kernel(Args a) {
  const uint64_t nchunks = (a.nbytes + 15) / 16;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t o = c * 16;
    uint8_t *p = a.dst + o;
    if (o + 16 <= a.nbytes && ((uintptr_t)p & 15u) == 0) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        uint32_t x = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) x |= (uint32_t)make_byte(a, a.start + o + 4 * q + b) << (8 * b);
        w[q] = x;
      }
      *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      const uint64_t n = (a.nbytes - o) < 16 ? (a.nbytes - o) : 16;
      for (uint64_t b = 0; b < n; b++) p[b] = make_byte(a, a.start + o + b);
    }
  }
}

int launch(const Args &a, void *stream) {
  if (a.nbytes == 0) return 0;
  if (!a.dst) return -1;
  const uint64_t nchunks = (a.nbytes + 15) / 16;
  uint64_t grid = (nchunks + 255) / 256;
  if (grid > 152ull * 64) grid = 152ull * 64;
  synth_kernel<<<(unsigned)grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
  if (cudaGetLastError() != cudaSuccess) return -3;
  return 0;
}

}  // namespace

extern "C" {

int pospop_synth_random(void *dst, size_t nbytes, uint64_t seed, uint64_t start, void *stream) {
  Args a{};
  a.dst = static_cast<uint8_t *>(dst);
  a.nbytes = nbytes;
  a.seed = seed;
  a.start = start;
  a.kind = kRandom;
  return launch(a, stream);
}

int pospop_synth_bernoulli(void *dst, size_t nbytes, uint64_t seed, uint64_t threshold,
                           uint64_t start, void *stream) {
  if (threshold > (1ull << 32)) return -1;
  Args a{};
  a.dst = static_cast<uint8_t *>(dst);
  a.nbytes = nbytes;
  a.seed = seed;
  a.start = start;
  a.threshold = threshold;
  a.kind = kBernoulli;
  return launch(a, stream);
}

int pospop_synth_one_hot(void *dst, size_t nbytes, uint64_t seed, const uint32_t *thresholds,
                         int k_minus_1, uint64_t start, void *stream) {
  if (k_minus_1 < 0 || k_minus_1 > 7 || (k_minus_1 > 0 && !thresholds)) return -1;
  Args a{};
  a.dst = static_cast<uint8_t *>(dst);
  a.nbytes = nbytes;
  a.seed = seed;
  a.start = start;
  a.kind = kOneHot;
  a.nth = k_minus_1;
  for (int t = 0; t < k_minus_1; t++) a.th[t] = thresholds[t];
  return launch(a, stream);
}

int pospop_synth_fill(void *dst, size_t nbytes, uint8_t value, void *stream) {
  Args a{};
  a.dst = static_cast<uint8_t *>(dst);
  a.nbytes = nbytes;
  a.kind = kFill;
  a.value = value;
  return launch(a, stream);
}

}  // extern "C"

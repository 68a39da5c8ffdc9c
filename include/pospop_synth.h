/*
 * pospop_synth.h -- C ABI of libpospop_synth.so, the device twin of the
 * seeded input generator (paper_2412_16370_gb300/synth.py).
 *
 * This library makes synthetic INPUTS for tests and benchmarks; it holds no
 * part of the counting method and the paper has no counterpart to it.  It
 * exists because multi-GiB inputs are generated far faster on the device.
 * Every function writes bytes [start, start + nbytes) of a SplitMix64-based
 * stream (G. L. Steele, D. Lea, C. H. Flood, OOPSLA 2014; output i of
 * stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15)), identical
 * byte for byte to the Python recipe of the same name.
 *
 * `dst` is a device pointer of the current device (any alignment), `stream`
 * a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 * asynchronous.  Return 0 on success, -1 for a bad argument, -3 if a launch
 * failed.
 */
#ifndef POSPOP_SYNTH_H
#define POSPOP_SYNTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Raw stream: byte k is byte k % 8 (little-endian) of output k / 8. */
int pospop_synth_random(void *dst, size_t nbytes, uint64_t seed, uint64_t start, void *stream);

/* Bit b of byte k is set iff (output(8k + b) >> 32) < threshold, threshold in
 * [0, 2^32] (P(bit) = threshold / 2^32). */
int pospop_synth_bernoulli(void *dst, size_t nbytes, uint64_t seed, uint64_t threshold,
                           uint64_t start, void *stream);

/* One-hot bytes: byte k = 1 << c, c = number of the k_minus_1 ascending
 * thresholds (host array) that are <= (output(k) >> 32); k_minus_1 <= 7. */
int pospop_synth_one_hot(void *dst, size_t nbytes, uint64_t seed, const uint32_t *thresholds,
                         int k_minus_1, uint64_t start, void *stream);

/* Every byte set to `value`. */
int pospop_synth_fill(void *dst, size_t nbytes, uint8_t value, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* POSPOP_SYNTH_H */

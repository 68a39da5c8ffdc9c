/*
 * pospopcnt_oracle.c -- CPU oracle for the positional population count.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline / reference leg may load this
 * library.  It shares no code, header, table or constant with the CUDA
 * path, and the CUDA path never loads it.
 *
 * What it computes (Clausecker, Lemire, Schintke, "Faster Positional-
 * Population Counts for AVX2, AVX-512, and ASIMD", arXiv 2412.16370):
 *
 *   - Fig. 2, the pseudo-C definition: for every word i < n and every bit
 *     position j < w, counts[j] += (words[i] >> j) & 1.  The counts are ADDED
 *     to what the caller passes in (Section 4, step 1 and its footnote:
 *     clearing C is optional).  oracle_pospop_u8/u16/u32/u64 are that loop,
 *     one per word width.
 *
 *   - Section 1 (introduction): the bit stream is viewed as w interleaved
 *     streams and the bits at positions j, j+w, j+2w, ... are summed.
 *     oracle_pospop_bytes is that definition on a little-endian byte stream:
 *     bit b of byte k is stream bit 8k+b and goes to counter (8k+b) mod w.
 *     For whole words this equals Fig. 2 read little-endian; a trailing
 *     partial word behaves as if zero-padded.  It also accepts w = 1, 2, 4
 *     (w = 1 is the conventional population count, Section 3.3) and the
 *     wider folds w = 128, 256.
 *
 *   - oracle_pospop_batch: the same definition over many arrays given by
 *     CSR byte offsets (one counts row of w entries per array).
 *
 *   - oracle_pospop_gather: several separate regions counted into ONE
 *     counter array, each region its own word stream (Section 4, step 1
 *     footnote: leaving C uncleared lets non-contiguous memory regions be
 *     counted together).
 *
 *   - oracle_pospop_masked: Fig. 2 restricted to the words whose bit in a
 *     selection bitmap is set (bit i of the bitmap, least significant bit
 *     of byte i/8 first, selects word i): the GROUP BY count of Section 1
 *     with a WHERE filter.
 *
 *   - oracle_pospop_bytes_mt: the timed CPU baseline.  It splits the input
 *     at word boundaries across threads and sums the per-thread counts,
 *     which is exact because the counts of a concatenation of whole words
 *     are the sums of the parts' counts.
 *
 * Build: gcc -O2 -fno-tree-vectorize -fPIC -shared -pthread (the paper's
 * scalar baseline was likewise compiled with auto-vectorisation inhibited,
 * Section 5).  The code is plain C99 and endian-neutral: words are assembled
 * from bytes with shifts, never by reinterpreting memory.
 *
 * Planted mistakes: when compiled with -DORACLE_MUTANT=k (k >= 1) one
 * deliberate error is compiled in so that the test suite can show that its
 * pins catch it.  The default build (ORACLE_MUTANT undefined or 0) has none.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* ------------------------------------------------------------------------
 * Fig. 2, one function per word width.  The typed arrays are read as
 * machine words; the paper's platforms are all little-endian, and so are the
 * machines this is built for.
 * ---------------------------------------------------------------------- */

void oracle_pospop_u8(uint64_t counts[8], const uint8_t *words, size_t n)
{
    for (size_t i = 0; i < n; i++)
        for (size_t j = 0; j < 8; j++)
            counts[j] += (words[i] >> j) & 1u;
}

void oracle_pospop_u16(uint64_t counts[16], const uint16_t *words, size_t n)
{
    for (size_t i = 0; i < n; i++)
        for (size_t j = 0; j < 16; j++)
            counts[j] += (uint64_t)((words[i] >> j) & 1u);
}

void oracle_pospop_u32(uint64_t counts[32], const uint32_t *words, size_t n)
{
    for (size_t i = 0; i < n; i++)
        for (size_t j = 0; j < 32; j++)
            counts[j] += (uint64_t)((words[i] >> j) & 1u);
}

void oracle_pospop_u64(uint64_t counts[64], const uint64_t *words, size_t n)
{
    for (size_t i = 0; i < n; i++)
        for (size_t j = 0; j < 64; j++)
            counts[j] += (words[i] >> j) & 1u;
}

/* ------------------------------------------------------------------------
 * Section 1: w interleaved bit streams over a byte stream.
 * ---------------------------------------------------------------------- */

/* Any power of two from 1 to 256: the interleaved-streams definition holds
 * for every w, and Section 4 states the algorithm for a general maximum word
 * size (the paper's code fixes it at 64). */
static int valid_w(int w)
{
    return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64 ||
           w == 128 || w == 256;
}

/* Counts of one byte stream, added into counts[0..w-1].  Stream bit q = 8k+b
 * (bit b of byte k, least significant bit first) is summed into counter
 * q mod w; w is a power of two, so q mod w is q & (w - 1). */
static void stream_counts(int w, uint64_t *counts, const uint8_t *bytes, size_t nbytes)
{
    const uint64_t wmask = (uint64_t)w - 1u;
    size_t k_end = nbytes;
#if ORACLE_MUTANT == 2
    /* planted: a trailing partial word is dropped instead of zero-padded */
    {
        size_t W = (w >= 8) ? (size_t)(w / 8) : 1;
        k_end = nbytes - nbytes % W;
    }
#endif
    for (size_t k = 0; k < k_end; k++) {
        unsigned byte = bytes[k];
#if ORACLE_MUTANT == 4
        /* planted: the last byte of the stream is skipped */
        if (k + 1 == nbytes) continue;
#endif
        for (unsigned b = 0; b < 8; b++) {
            uint64_t q = 8u * (uint64_t)k + b;
#if ORACLE_MUTANT == 1
            /* planted: big-endian word reading (byte order within a word reversed) */
            if (w >= 16) {
                uint64_t W = (uint64_t)w / 8u, kw = k % W;
                q = 8u * ((uint64_t)k - kw + (W - 1u - kw)) + b;
            }
#endif
            size_t j = (size_t)(q & wmask);
#if ORACLE_MUTANT == 3
            /* planted: position index off by one */
            j = (size_t)((j + 1u) & wmask);
#endif
            counts[j] += (byte >> b) & 1u;
        }
    }
}

int oracle_pospop_bytes(int w, uint64_t *counts, const uint8_t *bytes, size_t nbytes)
{
    if (!valid_w(w)) return ORACLE_EINVAL;
    if (nbytes == 0) return ORACLE_OK;
    if (counts == NULL || bytes == NULL) return ORACLE_EINVAL;
#if ORACLE_MUTANT == 5
    /* planted: counts are overwritten instead of added to */
    memset(counts, 0, sizeof(uint64_t) * (size_t)w);
#endif
    stream_counts(w, counts, bytes, nbytes);
    return ORACLE_OK;
}

int oracle_pospop_batch(int w, uint64_t *counts, const uint8_t *base,
                        const uint64_t *offsets, size_t m)
{
    if (!valid_w(w)) return ORACLE_EINVAL;
    if (m == 0) return ORACLE_OK;
    if (counts == NULL || offsets == NULL) return ORACLE_EINVAL;
    for (size_t a = 0; a < m; a++)
        if (offsets[a + 1] < offsets[a]) return ORACLE_EINVAL;
    for (size_t a = 0; a < m; a++) {
        size_t len = (size_t)(offsets[a + 1] - offsets[a]);
        if (len == 0) continue;
        if (base == NULL) return ORACLE_EINVAL;
        stream_counts(w, counts + (size_t)w * a, base + offsets[a], len);
    }
    return ORACLE_OK;
}

int oracle_pospop_gather(int w, uint64_t *counts, const uint64_t *ptrs, const uint64_t *lens,
                         size_t n)
{
    if (!valid_w(w)) return ORACLE_EINVAL;
    if (n == 0) return ORACLE_OK;
    if (counts == NULL || ptrs == NULL || lens == NULL) return ORACLE_EINVAL;
    for (size_t r = 0; r < n; r++)
        if (lens[r] > 0 && ptrs[r] == 0) return ORACLE_EINVAL;
#if ORACLE_MUTANT == 7
    /* planted: the regions are counted as one continuous stream (bit
     * positions carry over from one region to the next) */
    {
        uint64_t q0 = 0;
        for (size_t r = 0; r < n; r++) {
            const uint8_t *b = (const uint8_t *)(uintptr_t)ptrs[r];
            for (uint64_t k = 0; k < lens[r]; k++)
                for (unsigned bit = 0; bit < 8; bit++)
                    counts[(q0 + 8u * k + bit) & ((uint64_t)w - 1u)] += (b[k] >> bit) & 1u;
            q0 += 8u * lens[r];
        }
        return ORACLE_OK;
    }
#endif
    for (size_t r = 0; r < n; r++)
        if (lens[r] > 0)
            stream_counts(w, counts, (const uint8_t *)(uintptr_t)ptrs[r], (size_t)lens[r]);
    return ORACLE_OK;
}

int oracle_pospop_masked(int w, uint64_t *counts, const uint8_t *words, size_t n,
                         const uint8_t *mask)
{
    if (!(w == 8 || w == 16 || w == 32 || w == 64)) return ORACLE_EINVAL;
    if (n == 0) return ORACLE_OK;
    if (counts == NULL || words == NULL || mask == NULL) return ORACLE_EINVAL;
    size_t W = (size_t)w / 8;
    for (size_t i = 0; i < n; i++) {
        unsigned sel = (mask[i / 8] >> (i % 8)) & 1u;
#if ORACLE_MUTANT == 6
        /* planted: selection bits read most significant bit first */
        sel = (mask[i / 8] >> (7 - i % 8)) & 1u;
#endif
        if (sel == 0) continue;
        uint64_t v = 0;
        for (size_t k = 0; k < W; k++) v |= (uint64_t)words[i * W + k] << (8u * k);
        for (int j = 0; j < w; j++) counts[j] += (v >> j) & 1u;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Timed CPU baseline: the same definition split across threads at word
 * boundaries (additivity of the counts under concatenation).
 * ---------------------------------------------------------------------- */

struct mt_job {
    int w;
    const uint8_t *bytes;
    size_t nbytes;
    uint64_t counts[256];
};

/* Fig. 2 on little-endian words assembled from the byte stream; a trailing
 * partial word is zero-padded.  For w < 8 a byte is one 8-bit word whose
 * bit j is counted in counter j mod w. */
static void fig2_word_loop(int w, uint64_t *counts, const uint8_t *bytes, size_t nbytes)
{
    size_t W = (w >= 8) ? (size_t)(w / 8) : 1;
    unsigned bits = (w >= 8) ? (unsigned)w : 8u;
    size_t nwords = (nbytes + W - 1) / W;
    for (size_t i = 0; i < nwords; i++) {
        if (w <= 64) {
            uint64_t v = 0;
            for (size_t k = 0; k < W && i * W + k < nbytes; k++)
                v |= (uint64_t)bytes[i * W + k] << (8u * k);
            for (unsigned j = 0; j < bits; j++)
                counts[j & (unsigned)(w - 1)] += (v >> j) & 1u;
        } else {
            /* a 128- or 256-bit word: bit j is bit j % 8 of its byte j / 8 */
            for (unsigned j = 0; j < bits; j++) {
                size_t k = i * W + j / 8;
                if (k < nbytes) counts[j] += (bytes[k] >> (j % 8)) & 1u;
            }
        }
    }
}

static void *mt_worker(void *arg)
{
    struct mt_job *job = (struct mt_job *)arg;
    memset(job->counts, 0, sizeof(job->counts));
    if (job->nbytes) fig2_word_loop(job->w, job->counts, job->bytes, job->nbytes);
    return NULL;
}

int oracle_pospop_bytes_mt(int w, uint64_t *counts, const uint8_t *bytes, size_t nbytes,
                           int nthreads)
{
    if (!valid_w(w)) return ORACLE_EINVAL;
    if (nbytes == 0) return ORACLE_OK;
    if (counts == NULL || bytes == NULL) return ORACLE_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    size_t W = (w >= 8) ? (size_t)(w / 8) : 1;
    size_t nwords = (nbytes + W - 1) / W;
    if ((size_t)nthreads > nwords) nthreads = (int)nwords;

    struct mt_job *jobs = (struct mt_job *)calloc((size_t)nthreads, sizeof(struct mt_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return ORACLE_EINVAL; }

    size_t per = nwords / (size_t)nthreads, extra = nwords % (size_t)nthreads, wstart = 0;
    for (int t = 0; t < nthreads; t++) {
        size_t wcount = per + ((size_t)t < extra ? 1 : 0);
        size_t b0 = wstart * W, b1 = (wstart + wcount) * W;
        if (b1 > nbytes) b1 = nbytes;
        jobs[t].w = w;
        jobs[t].bytes = bytes + b0;
        jobs[t].nbytes = b1 - b0;
        wstart += wcount;
    }
    int started = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&tids[t], NULL, mt_worker, &jobs[t]) != 0) break;
        started = t;
    }
    mt_worker(&jobs[0]);
    for (int t = 1; t <= started; t++) pthread_join(tids[t], NULL);
    for (int t = started + 1; t < nthreads; t++) mt_worker(&jobs[t]); /* threads that failed to start */
    for (int t = 0; t < nthreads; t++)
        for (int j = 0; j < w; j++) counts[j] += jobs[t].counts[j];
    free(jobs);
    free(tids);
    return ORACLE_OK;
}

/* Build identity, so a test can tell a mutant build from the default one. */
int oracle_mutant_id(void) { return ORACLE_MUTANT; }

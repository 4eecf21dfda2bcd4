/*
 * Multithreaded generator of batches of uniform random DFAs (inputs only; none of the
 * minimization arithmetic).  Same streams as inputs.random_dfa: element j of DFA i's delta is
 * bounded(splitmix64(sub_delta[i], j), n_i) and state s accepts iff
 * (splitmix64(sub_acc[i], s) >> 11) < thr[i]; the per-DFA stream seeds and thresholds are
 * computed by the caller (inputs.py) so that both sides share one definition of them.
 *
 * splitmix64: value j of a stream with seed x is the finalizer of x + (j + 1) * 0x9E3779B97F4A7C15
 * (Steele, Lea & Flood 2014); bounded(x, m) is the high 64 bits of x * m (Lemire).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

static inline uint64_t fin(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream(uint64_t seed, uint64_t j)
{
    return fin(seed + (j + 1) * 0x9E3779B97F4A7C15ULL);
}

static inline uint32_t bounded(uint64_t x, uint64_t m)
{
    return (uint32_t)(((unsigned __int128)x * m) >> 64);
}

typedef struct {
    int32_t count;
    const int64_t *state_off;   /* [count+1] */
    const int64_t *delta_off;   /* [count+1] */
    const int32_t *k;
    const uint64_t *sub_delta, *sub_acc, *thr;
    int32_t *delta;
    uint32_t *accept;
    int64_t e0, e1;             /* delta elements of this worker */
    int64_t w0, w1;             /* accept words of this worker */
} job_t;

/* last DFA whose offset <= x */
static int32_t find(const int64_t *off, int32_t count, int64_t x)
{
    int32_t lo = 0, hi = count - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) / 2;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

static void *work(void *arg)
{
    job_t *J = (job_t *)arg;
    if (J->e0 < J->e1) {
        int32_t i = find(J->delta_off, J->count, J->e0);
        for (int64_t e = J->e0; e < J->e1; ++e) {
            while (e >= J->delta_off[i + 1]) ++i;
            const int64_t n = J->state_off[i + 1] - J->state_off[i];
            J->delta[e] = (int32_t)bounded(stream(J->sub_delta[i], (uint64_t)(e - J->delta_off[i])),
                                           (uint64_t)n);
        }
    }
    const int64_t total = J->state_off[J->count];
    if (J->w0 < J->w1) {
        int32_t i = find(J->state_off, J->count, J->w0 * 32);
        for (int64_t w = J->w0; w < J->w1; ++w) {
            uint32_t word = 0;
            for (int b = 0; b < 32; ++b) {
                const int64_t g = w * 32 + b;
                if (g >= total) break;
                while (g >= J->state_off[i + 1]) ++i;
                const uint64_t x = stream(J->sub_acc[i], (uint64_t)(g - J->state_off[i]));
                if ((x >> 11) < J->thr[i]) word |= 1u << b;
            }
            J->accept[w] = word;
        }
    }
    return NULL;
}

int inputs_random_batch(int32_t count, const int64_t *state_off, const int64_t *delta_off,
                        const int32_t *k, const uint64_t *sub_delta, const uint64_t *sub_acc,
                        const uint64_t *thr, int32_t *delta, uint32_t *accept, int32_t threads)
{
    if (count < 1 || threads < 1) return -1;
    (void)k;
    const int64_t E = delta_off[count], W = (state_off[count] + 31) / 32;
    job_t *jobs = (job_t *)calloc((size_t)threads, sizeof(job_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return -2; }
    for (int t = 0; t < threads; ++t) {
        job_t *J = &jobs[t];
        J->count = count; J->state_off = state_off; J->delta_off = delta_off; J->k = k;
        J->sub_delta = sub_delta; J->sub_acc = sub_acc; J->thr = thr;
        J->delta = delta; J->accept = accept;
        J->e0 = E * t / threads; J->e1 = E * (t + 1) / threads;
        J->w0 = W * t / threads; J->w1 = W * (t + 1) / threads;
        pthread_create(&tid[t], NULL, work, J);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    return 0;
}

/*
 * Bit-splitter B_nbits (same definition as inputs.bitsplitter_dfa): state x is a bit string,
 * letter column m-1 (m = 1..nbits-1) maps x to (x with its low m+1 bits replaced by
 * (not bit m) followed by m zeros) if bit m-1 of x is 1, and to x otherwise.  delta is
 * state-major [2^nbits][nbits-1]; accept bit x is the top bit of x.
 */
typedef struct {
    int32_t nbits;
    int64_t x0, x1;
    int32_t *delta;
    uint32_t *accept;
} bits_job_t;

static void *bits_work(void *arg)
{
    const bits_job_t *J = (const bits_job_t *)arg;
    const int32_t k = J->nbits - 1;
    for (int64_t x = J->x0; x < J->x1; ++x) {
        int32_t *row = J->delta + x * k;
        for (int32_t m = 1; m <= k; ++m) {
            const int64_t low = ((int64_t)1 << (m + 1)) - 1;
            const int64_t b = (x >> m) & 1;
            row[m - 1] = ((x >> (m - 1)) & 1) ? (int32_t)((x & ~low) | ((1 - b) << m))
                                               : (int32_t)x;
        }
    }
    /* accept words owned by this worker: x0 and x1 are multiples of 32 except at the end */
    for (int64_t w = J->x0 / 32; w < (J->x1 + 31) / 32; ++w) {
        uint32_t v = 0;
        for (int j = 0; j < 32; ++j) {
            const int64_t x = w * 32 + j;
            if (x < ((int64_t)1 << J->nbits) && ((x >> (J->nbits - 1)) & 1)) v |= 1u << j;
        }
        J->accept[w] = v;
    }
    return NULL;
}

int inputs_bitsplitter(int32_t nbits, int32_t *delta, uint32_t *accept, int32_t threads)
{
    if (nbits < 2 || nbits > 30 || threads < 1) return -1;
    const int64_t n = (int64_t)1 << nbits;
    bits_job_t *jobs = (bits_job_t *)calloc((size_t)threads, sizeof(bits_job_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return -2; }
    for (int t = 0; t < threads; ++t) {
        bits_job_t *J = &jobs[t];
        J->nbits = nbits;
        J->x0 = (n / 32) * t / threads * 32;
        J->x1 = t + 1 == threads ? n : (n / 32) * (t + 1) / threads * 32;
        J->delta = delta;
        J->accept = accept;
        pthread_create(&tid[t], NULL, bits_work, J);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    return 0;
}

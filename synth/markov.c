/*
 * Seeded synthetic DNA text: an order-2 Markov chain over {A, C, G, T}.
 *
 * Input generator shared by the tests, the oracle and the CUDA path.  It
 * holds none of the matching method's arithmetic: it only writes ASCII.
 *
 * Reproducibility: the text is cut into blocks of SYNTH_BLOCK bases; block b
 * draws its random numbers from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) keyed by (seed, b),
 * so the output does not depend on the thread count.  Each block starts its
 * chain from two letters drawn uniformly.
 *
 * thresholds: 16 contexts (4*x[t-2] + x[t-1], letters in A,C,G,T order) times
 * 3 cumulative thresholds on a 32-bit scale; the next letter is the number of
 * thresholds that a uniform 32-bit draw reaches.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#define SYNTH_BLOCK (1u << 20)

static inline uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

typedef struct {
    uint8_t *out;
    uint64_t start, end, seed;
    const uint32_t *thr;
    uint64_t b0, b1;
} job_t;

/* Runs block b's chain and stores the symbols whose global index lies in
 * [start, end) at out[index - start]. */
static void gen_block(uint8_t *out, uint64_t start, uint64_t end, uint64_t seed,
                      const uint32_t *thr, uint64_t b)
{
    static const uint8_t letters[4] = {'A', 'C', 'G', 'T'};
    uint64_t i = b * (uint64_t)SYNTH_BLOCK;
    uint64_t stop = i + SYNTH_BLOCK;
    if (stop > end) stop = end;
    uint64_t key = splitmix64(seed ^ splitmix64(b + 0x5851f42d4c957f2dull));
    uint64_t ctr = 0;
    uint64_t r = splitmix64(key + ctr++);
    unsigned x2 = (unsigned)(r & 3), x1 = (unsigned)((r >> 2) & 3);
    if (i < stop) { if (i >= start) out[i - start] = letters[x2]; ++i; }
    if (i < stop) { if (i >= start) out[i - start] = letters[x1]; ++i; }
    while (i < stop) {
        uint64_t w = splitmix64(key + ctr++);
        for (int h = 0; h < 2 && i < stop; ++h) {
            uint32_t u = (uint32_t)(h ? (w >> 32) : w);
            const uint32_t *t = thr + 3 * (4 * x2 + x1);
            unsigned x = (u >= t[0]) + (u >= t[1]) + (u >= t[2]);
            if (i >= start) out[i - start] = letters[x];
            ++i;
            x2 = x1;
            x1 = x;
        }
    }
}

static void *run(void *arg)
{
    job_t *j = (job_t *)arg;
    for (uint64_t b = j->b0; b < j->b1; ++b)
        gen_block(j->out, j->start, j->end, j->seed, j->thr, b);
    return NULL;
}

/* Symbols [start, start + len) of the text with the given seed. */
void synth_markov_range(uint8_t *out, uint64_t start, uint64_t len, uint64_t seed,
                        const uint32_t *thresholds, int nthreads)
{
    if (len == 0) return;
    uint64_t end = start + len;
    uint64_t bfirst = start / SYNTH_BLOCK, blast = (end - 1) / SYNTH_BLOCK + 1;
    uint64_t nb = blast - bfirst;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > nb) nthreads = (int)nb;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        for (uint64_t b = bfirst; b < blast; ++b) gen_block(out, start, end, seed, thresholds, b);
        free(jobs); free(th);
        return;
    }
    for (int q = 0; q < nthreads; ++q) {
        jobs[q].out = out; jobs[q].start = start; jobs[q].end = end;
        jobs[q].seed = seed; jobs[q].thr = thresholds;
        jobs[q].b0 = bfirst + nb * (uint64_t)q / (uint64_t)nthreads;
        jobs[q].b1 = bfirst + nb * (uint64_t)(q + 1) / (uint64_t)nthreads;
    }
    int started = 0;
    for (int q = 1; q < nthreads; ++q) {
        if (pthread_create(&th[q], NULL, run, &jobs[q]) != 0) break;
        started = q;
    }
    run(&jobs[0]);
    for (int q = started + 1; q < nthreads; ++q) run(&jobs[q]);
    for (int q = 1; q <= started; ++q) pthread_join(th[q], NULL);
    free(jobs); free(th);
}

void synth_markov(uint8_t *out, uint64_t n, uint64_t seed,
                  const uint32_t *thresholds, int nthreads)
{
    synth_markov_range(out, 0, n, seed, thresholds, nthreads);
}

/* GC fraction of a text (counts C and G), for calibration checks. */
double synth_gc_fraction(const uint8_t *txt, uint64_t n)
{
    uint64_t gc = 0;
    for (uint64_t i = 0; i < n; ++i) gc += (txt[i] == 'C') | (txt[i] == 'G');
    return n ? (double)gc / (double)n : 0.0;
}

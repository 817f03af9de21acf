/*
 * rmat.c -- seeded synthetic inputs shared by the tests, the smoke check and
 * the benchmark.  It holds no PageRank arithmetic: only random numbers and
 * edge-list bookkeeping.
 *
 * Random numbers: a counter-based generator built from the SplitMix64
 * finaliser (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Every draw is a pure function of
 * (seed, stream, counter), so output does not depend on the thread count.
 *
 * R-MAT (D. Chakrabarti, Y. Zhan, C. Faloutsos, SDM 2004; the generator of
 * the Graph500 benchmark): each edge picks one quadrant of the adjacency
 * matrix per level with probabilities a, b, c, 1-a-b-c.  No per-level noise.
 * Vertex labels are then scrambled by a seeded bijection on [0, 2^scale).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z += GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* counter-based draw: a pure function of (seed, stream, counter) */
uint64_t gen_rand64(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return mix64(mix64(mix64(seed) ^ stream) ^ counter);
}

/* uniform double in [0, 1) with 53 random bits */
double gen_uniform(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (double)(gen_rand64(seed, stream, counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* streams (arbitrary distinct constants) */
#define STREAM_RMAT 0x524d4154ULL      /* quadrant draws */
#define STREAM_SCRAMBLE 0x5343524dULL  /* label bijection */
#define STREAM_SHUFFLE 0x53485546ULL   /* edge order */
#define STREAM_FIXUP 0x46495855ULL     /* dangling fix-up */

/* Seeded bijection on [0, 2^scale): composition of bijections (xor with a
 * constant, multiplication by an odd constant, xor-shift right), all mod
 * 2^scale. */
typedef struct { uint64_t mask, k[8]; int shift; } scrambler;

static void scrambler_init(scrambler *s, int scale, uint64_t seed)
{
    s->mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1ULL);
    for (int i = 0; i < 8; ++i) s->k[i] = gen_rand64(seed, STREAM_SCRAMBLE, (uint64_t)i);
    s->shift = scale > 1 ? (scale + 1) / 2 : 1;
}

static inline uint64_t scramble(const scrambler *s, uint64_t v)
{
    for (int r = 0; r < 4; ++r) {
        v = (v ^ s->k[2 * r]) & s->mask;
        v = (v * (s->k[2 * r + 1] | 1ULL)) & s->mask;
        v ^= v >> s->shift;
    }
    return v & s->mask;
}

typedef struct {
    int scale, do_scramble;
    uint64_t seed, t_a, t_ab, t_abc;
    int64_t begin, end;
    int32_t *src, *dst;
    const scrambler *scr;
} rmat_job;

static void *rmat_worker(void *arg)
{
    rmat_job *j = (rmat_job *)arg;
    for (int64_t e = j->begin; e < j->end; ++e) {
        uint64_t u = 0, v = 0;
        uint64_t bits = 0;
        for (int l = 0; l < j->scale; ++l) {
            if ((l & 1) == 0) bits = gen_rand64(j->seed, STREAM_RMAT, (uint64_t)e * 64u + (uint64_t)l);
            uint64_t r = (l & 1) ? (bits >> 32) : (bits & 0xffffffffULL);
            uint64_t bit = 1ULL << (j->scale - 1 - l);
            if (r < j->t_a) {
            } else if (r < j->t_ab) {
                v |= bit;
            } else if (r < j->t_abc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
        if (j->do_scramble) {
            u = scramble(j->scr, u);
            v = scramble(j->scr, v);
        }
        j->src[e] = (int32_t)u;
        j->dst[e] = (int32_t)v;
    }
    return NULL;
}

static int nthreads_for(int64_t m, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 64) threads = 64;
    if (m < 100000) threads = 1;
    return threads;
}

/* Raw R-MAT edge list of m = ef * 2^scale edges (self-loops and duplicates
 * included), written to src/dst.  Quadrant probabilities are compared at
 * 32-bit resolution. */
int gen_rmat_raw(int scale, int64_t m, double a, double b, double c, uint64_t seed,
                 int do_scramble, int threads, int32_t *src, int32_t *dst)
{
    if (scale < 1 || scale > 30 || m < 0) return 1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
    scrambler scr;
    scrambler_init(&scr, scale, seed);
    const double two32 = 4294967296.0;
    uint64_t t_a = (uint64_t)(a * two32);
    uint64_t t_ab = (uint64_t)((a + b) * two32);
    uint64_t t_abc = (uint64_t)((a + b + c) * two32);
    int nt = nthreads_for(m, threads);
    pthread_t tid[64];
    rmat_job jobs[64];
    for (int t = 0; t < nt; ++t) {
        rmat_job *j = &jobs[t];
        j->scale = scale;
        j->do_scramble = do_scramble;
        j->seed = seed;
        j->t_a = t_a;
        j->t_ab = t_ab;
        j->t_abc = t_abc;
        j->begin = m * t / nt;
        j->end = m * (t + 1) / nt;
        j->src = src;
        j->dst = dst;
        j->scr = &scr;
        if (nt == 1) rmat_worker(j);
        else pthread_create(&tid[t], NULL, rmat_worker, j);
    }
    if (nt > 1)
        for (int t = 0; t < nt; ++t) pthread_join(tid[t], NULL);
    return 0;
}

/* LSD radix sort of (key, id) pairs by key over the low `bits` bits, 11 bits
 * per pass (stable). */
static int radix_sort_pairs(int64_t m, int bits, uint64_t *key, uint32_t *id)
{
    uint64_t *k2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    uint32_t *i2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 2049);
    if (!k2 || !i2 || !cnt) { free(k2); free(i2); free(cnt); return 2; }
    for (int sh = 0; sh < bits; sh += 11) {
        memset(cnt, 0, sizeof(int64_t) * 2049);
        for (int64_t i = 0; i < m; ++i) cnt[((key[i] >> sh) & 0x7ff) + 1]++;
        for (int k = 0; k < 2048; ++k) cnt[k + 1] += cnt[k];
        for (int64_t i = 0; i < m; ++i) {
            int64_t p = cnt[(key[i] >> sh) & 0x7ff]++;
            k2[p] = key[i];
            i2[p] = id[i];
        }
        memcpy(key, k2, sizeof(uint64_t) * (size_t)m);
        memcpy(id, i2, sizeof(uint32_t) * (size_t)m);
    }
    free(k2);
    free(i2);
    free(cnt);
    return 0;
}

/* Removes self-loops and repeated (src, dst) pairs in place, keeping the
 * first occurrence of each pair and the original order of the survivors.
 * Returns the new edge count (or -1 on allocation failure). */
int64_t gen_dedup(int scale, int64_t m, int32_t *src, int32_t *dst)
{
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    uint32_t *id = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    uint8_t *keep = (uint8_t *)calloc((size_t)(m > 0 ? m : 1), 1);
    if (!key || !id || !keep) { free(key); free(id); free(keep); return -1; }
    for (int64_t e = 0; e < m; ++e) {
        key[e] = ((uint64_t)(uint32_t)src[e] << scale) | (uint64_t)(uint32_t)dst[e];
        id[e] = (uint32_t)e;
    }
    if (radix_sort_pairs(m, 2 * scale, key, id)) { free(key); free(id); free(keep); return -1; }
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        uint32_t e = id[i];
        if (src[e] != dst[e]) keep[e] = 1;
    }
    int64_t w = 0;
    for (int64_t e = 0; e < m; ++e)
        if (keep[e]) {
            src[w] = src[e];
            dst[w] = dst[e];
            ++w;
        }
    free(key);
    free(id);
    free(keep);
    return w;
}

/* Seeded Fisher-Yates shuffle of the edge order. */
void gen_shuffle(int64_t m, uint64_t seed, int32_t *src, int32_t *dst)
{
    for (int64_t i = m - 1; i > 0; --i) {
        uint64_t r = gen_rand64(seed, STREAM_SHUFFLE, (uint64_t)i);
        int64_t j = (int64_t)(r % (uint64_t)(i + 1));
        int32_t t = src[i]; src[i] = src[j]; src[j] = t;
        t = dst[i]; dst[i] = dst[j]; dst[j] = t;
    }
}

/*
 * Makes exactly `target` vertices dangling (out-degree 0).  Too many
 * dangling: a seeded choice of the excess gets one out-edge each to a
 * uniform random other vertex (appended at the end; cannot duplicate an
 * existing edge since the vertex had none).  Too few: a seeded choice of
 * non-dangling vertices loses all out-edges.  `cap` is the capacity of
 * src/dst.  Returns the new edge count, or -1 if capacity or memory is short.
 */
int64_t gen_fix_dangling(int32_t n, int64_t m, int64_t cap, int64_t target, uint64_t seed,
                         int32_t *src, int32_t *dst)
{
    if (target < 0 || target > n || n < 2) return -1;
    int32_t *deg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!deg) return -1;
    for (int64_t e = 0; e < m; ++e) deg[src[e]]++;
    int64_t dang = 0;
    for (int32_t u = 0; u < n; ++u) dang += deg[u] == 0;
    /* seeded order of candidate vertices: sort by a random key */
    int want_dangling = dang < target; /* candidates are non-dangling */
    int64_t ncand = want_dangling ? (n - dang) : dang;
    int64_t need = want_dangling ? (target - dang) : (dang - target);
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ncand > 0 ? ncand : 1));
    uint32_t *id = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(ncand > 0 ? ncand : 1));
    if (!key || !id) { free(deg); free(key); free(id); return -1; }
    int64_t k = 0;
    for (int32_t u = 0; u < n; ++u) {
        int is_dang = deg[u] == 0;
        if (is_dang != want_dangling) {
            key[k] = gen_rand64(seed, STREAM_FIXUP, (uint64_t)u) >> 1;
            id[k] = (uint32_t)u;
            ++k;
        }
    }
    radix_sort_pairs(ncand, 64, key, id);
    int64_t out = m;
    if (!want_dangling) {
        if (m + need > cap) { free(deg); free(key); free(id); return -1; }
        for (int64_t i = 0; i < need; ++i) {
            int32_t u = (int32_t)id[i];
            uint64_t r = gen_rand64(seed, STREAM_FIXUP ^ 0xffffULL, (uint64_t)u);
            int32_t v = (int32_t)(r % (uint64_t)(n - 1));
            if (v >= u) v += 1;
            src[out] = u;
            dst[out] = v;
            ++out;
        }
    } else {
        uint8_t *drop = (uint8_t *)calloc((size_t)n, 1);
        if (!drop) { free(deg); free(key); free(id); return -1; }
        for (int64_t i = 0; i < need; ++i) drop[id[i]] = 1;
        int64_t w = 0;
        for (int64_t e = 0; e < m; ++e)
            if (!drop[src[e]]) {
                src[w] = src[e];
                dst[w] = dst[e];
                ++w;
            }
        out = w;
        free(drop);
    }
    free(deg);
    free(key);
    free(id);
    return out;
}

/* n uniform doubles in [0, 1) from one stream (weights, coefficients). */
void gen_uniform_array(int64_t n, uint64_t seed, uint64_t stream, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = gen_uniform(seed, stream, (uint64_t)i);
}

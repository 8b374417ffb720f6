/*
 * Seeded synthetic-input generators for ByteStore workloads.
 *
 * This file draws random numbers and maps them to int32 column values. It holds
 * none of the storage method's arithmetic (no dictionary, no prefix-preserving
 * code, no layout, no predicate): both the CPU oracle's tests and the GPU path
 * call it to obtain identical inputs.
 *
 * Generators (all counter-based, so any index range can be produced in any
 * order by any number of threads and the output never depends on the thread
 * count):
 *   - SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) output function applied to
 *     key + (i + 1) * golden-gamma gives the i-th 64-bit draw of a stream.
 *   - Zipf(s) over ranks 1..N: inverse CDF with a guide table (Chen & Asau 1974)
 *     for N <= 2^24; rejection-inversion (Hoermann & Derflinger 1996) above.
 *   - A 4-round balanced Feistel network on d bits (cycle-walking for odd d)
 *     as a seeded bijection of [0, 2^d), used to map Zipf ranks to values.
 *
 * Built with -ffp-contract=off so no multiply-add is fused differently on
 * x86-64 and AArch64 hosts.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm64_mix(seed * GOLDEN_GAMMA + sm64_mix(stream + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return sm64_mix(key + (i + 1) * GOLDEN_GAMMA); }

static inline double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------ threads */
typedef void (*range_fn)(void *ctx, uint64_t begin, uint64_t end);
typedef struct { range_fn fn; void *ctx; uint64_t b, e; } range_job;

static void *range_thread(void *p) {
    range_job *j = (range_job *)p;
    j->fn(j->ctx, j->b, j->e);
    return NULL;
}

static void parallel_range(range_fn fn, void *ctx, uint64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > n / 65536 + 1) nthreads = (int)(n / 65536 + 1);
    if (nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    range_job jobs[256];
    uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    for (int t = 0; t < nthreads; t++) {
        uint64_t b = chunk * (uint64_t)t, e = b + chunk;
        if (b > n) b = n;
        if (e > n) e = n;
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].b = b; jobs[t].e = e;
        if (pthread_create(&th[t], NULL, range_thread, &jobs[t]) != 0) {
            fn(ctx, b, e);
            th[t] = 0;
        }
    }
    for (int t = 0; t < nthreads; t++)
        if (th[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------ raw uint64 */
typedef struct { uint64_t key, start; uint64_t *out; } u64_ctx;
static void u64_range(void *p, uint64_t b, uint64_t e) {
    u64_ctx *c = (u64_ctx *)p;
    for (uint64_t i = b; i < e; i++) c->out[i] = draw(c->key, c->start + i);
}

void synth_u64(uint64_t seed, uint64_t stream, uint64_t start, uint64_t n, uint64_t *out, int nthreads) {
    u64_ctx c = {stream_key(seed, stream), start, out};
    parallel_range(u64_range, &c, n, nthreads);
}

/* ------------------------------------------------------------------ Zipf */
/* Zipf(s) over ranks r = 1..N with P(r) proportional to r^-s. Output is the
 * 0-based rank r - 1 (0 = most frequent). s == 0 is the uniform distribution. */

typedef struct {
    uint64_t key, N;
    uint64_t start;  /* out[i] is row start + i of the stream */
    double s;
    /* inverse-CDF path */
    const double *cdf;
    const uint32_t *guide;
    uint64_t G;
    /* rejection-inversion path */
    double h_lo, h_hi;
    uint32_t *out;
} zipf_ctx;

static double zH(double x, double s) {
    /* integral of t^-s: log(x) for s == 1, (x^(1-s) - 1)/(1-s) otherwise,
     * written with expm1 so s close to 1 keeps its precision */
    double lx = log(x);
    double a = (1.0 - s) * lx;
    if (fabs(a) < 1e-12) return lx;
    return expm1(a) / (1.0 - s);
}

static double zHinv(double u, double s) {
    double a = (1.0 - s) * u;
    if (fabs(a) < 1e-12) return exp(u);
    return exp(log1p(a) / (1.0 - s));
}

static void zipf_uniform_range(void *p, uint64_t b, uint64_t e) {
    zipf_ctx *c = (zipf_ctx *)p;
    for (uint64_t i = b; i < e; i++) {
        uint64_t z = draw(c->key, c->start + i);
        /* high 64 bits of z * N: an index in [0, N) */
        unsigned __int128 m = (unsigned __int128)z * (unsigned __int128)c->N;
        c->out[i] = (uint32_t)(m >> 64);
    }
}

static void zipf_cdf_range(void *p, uint64_t b, uint64_t e) {
    zipf_ctx *c = (zipf_ctx *)p;
    for (uint64_t i = b; i < e; i++) {
        double u = u01(draw(c->key, c->start + i));
        uint64_t g = (uint64_t)(u * (double)c->G);
        if (g >= c->G) g = c->G - 1;
        uint64_t r = c->guide[g];
        while (r + 1 < c->N && c->cdf[r] <= u) r++;
        c->out[i] = (uint32_t)r;
    }
}

static void zipf_rejinv_range(void *p, uint64_t b, uint64_t e) {
    zipf_ctx *c = (zipf_ctx *)p;
    for (uint64_t i = b; i < e; i++) {
        for (uint64_t attempt = 0;; attempt++) {
            /* attempt t > 0 draws from its own derived stream */
            uint64_t key = attempt ? sm64_mix(c->key + attempt * 0xD1B54A32D192ED03ULL) : c->key;
            double u01v = u01(draw(key, c->start + i));
            double u = c->h_hi + u01v * (c->h_lo - c->h_hi);
            double x = zHinv(u, c->s);
            double kf = floor(x + 0.5);
            if (kf < 1.0) kf = 1.0;
            if (kf > (double)c->N) kf = (double)c->N;
            /* accept when u falls inside the bar of height h(k) that ends at k + 1/2 */
            if (u >= zH(kf + 0.5, c->s) - exp(-c->s * log(kf))) {
                c->out[i] = (uint32_t)((uint64_t)kf - 1);
                break;
            }
        }
    }
}

/* Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
/* Rows start .. start + n - 1 of the stream (row i depends on i alone, so a
 * column can be generated in disjoint pieces). */
int synth_zipf_at(uint64_t seed, uint64_t stream, uint64_t start, uint64_t n, uint64_t N, double s, uint32_t *out,
                  int nthreads) {
    if (N == 0 || N > 4294967296ULL || s < 0.0) return -1;
    zipf_ctx c;
    memset(&c, 0, sizeof c);
    c.key = stream_key(seed, stream);
    c.start = start;
    c.N = N;
    c.s = s;
    c.out = out;
    if (s == 0.0) {
        parallel_range(zipf_uniform_range, &c, n, nthreads);
        return 0;
    }
    if (N <= (1ULL << 24)) {
        double *cdf = (double *)malloc(sizeof(double) * N);
        uint64_t G = N < 1024 ? 1024 : N;
        uint32_t *guide = (uint32_t *)malloc(sizeof(uint32_t) * G);
        if (!cdf || !guide) { free(cdf); free(guide); return -2; }
        double acc = 0.0;
        for (uint64_t r = 0; r < N; r++) { acc += exp(-s * log((double)(r + 1))); cdf[r] = acc; }
        for (uint64_t r = 0; r < N; r++) cdf[r] /= acc;
        cdf[N - 1] = 1.0;
        uint64_t r = 0;
        for (uint64_t g = 0; g < G; g++) {
            double t = (double)g / (double)G;
            while (r + 1 < N && cdf[r] <= t) r++;
            guide[g] = (uint32_t)r;
        }
        c.cdf = cdf; c.guide = guide; c.G = G;
        parallel_range(zipf_cdf_range, &c, n, nthreads);
        free(cdf); free(guide);
        return 0;
    }
    c.h_lo = zH(1.5, s) - 1.0;
    c.h_hi = zH((double)N + 0.5, s);
    parallel_range(zipf_rejinv_range, &c, n, nthreads);
    return 0;
}

int synth_zipf(uint64_t seed, uint64_t stream, uint64_t n, uint64_t N, double s, uint32_t *out, int nthreads) {
    return synth_zipf_at(seed, stream, 0, n, N, s, out, nthreads);
}

/* --------------------------------------------------------------- Feistel */
typedef struct { int d; uint64_t key; const uint32_t *in; uint32_t *out; } feistel_ctx;

static inline uint64_t feistel_even(uint64_t x, int bits, uint64_t key) {
    int h = bits / 2;
    uint64_t mask = (h == 64) ? ~0ULL : ((1ULL << h) - 1);
    uint64_t L = (x >> h) & mask, R = x & mask;
    for (int round = 0; round < 4; round++) {
        uint64_t F = sm64_mix(R ^ (key + (uint64_t)round * GOLDEN_GAMMA)) & mask;
        uint64_t nL = R, nR = L ^ F;
        L = nL; R = nR;
    }
    return (L << h) | R;
}

static inline uint32_t feistel_perm(uint32_t x, int d, uint64_t key) {
    if (d == 0) return 0;
    int bits = (d & 1) ? d + 1 : d;
    uint64_t y = x;
    do { y = feistel_even(y, bits, key); } while (y >> d);
    return (uint32_t)y;
}

static void feistel_range(void *p, uint64_t b, uint64_t e) {
    feistel_ctx *c = (feistel_ctx *)p;
    for (uint64_t i = b; i < e; i++) c->out[i] = feistel_perm(c->in[i], c->d, c->key);
}

/* Seeded bijection of [0, 2^d), 1 <= d <= 32, applied elementwise. */
int synth_feistel(const uint32_t *in, uint64_t n, int d, uint64_t seed, uint32_t *out, int nthreads) {
    if (d < 0 || d > 32) return -1;
    feistel_ctx c = {d, stream_key(seed, 0xFE15E1ULL), in, out};
    parallel_range(feistel_range, &c, n, nthreads);
    return 0;
}

/* ---------------------------------------------------------------- gather */
typedef struct { const uint32_t *idx; const int32_t *table; int32_t *out; } gather_ctx;
static void gather_range(void *p, uint64_t b, uint64_t e) {
    gather_ctx *c = (gather_ctx *)p;
    for (uint64_t i = b; i < e; i++) c->out[i] = c->table[c->idx[i]];
}

/* out[i] = table[idx[i]] (idx must be in range; the caller checks). */
void synth_gather(const uint32_t *idx, uint64_t n, const int32_t *table, int32_t *out, int nthreads) {
    gather_ctx c = {idx, table, out};
    parallel_range(gather_range, &c, n, nthreads);
}

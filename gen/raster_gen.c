/*
 * Seeded synthetic point generator for RASTER workloads.
 *
 * This module holds no clustering arithmetic: it only draws points.  It is
 * the one piece of code that both the CPU oracle (tests) and the CUDA path
 * (tests, bench) consume, so that both see the same bytes.
 *
 * Workload shape (stands in for the paper's unavailable generator, Sect. 4.2
 * "Data": clusters of uniform points around random centres, randomly
 * shuffled): K square clusters of side 2*half_width whose centres are uniform
 * in [0, L)^2, followed by uniform noise on [0, L)^2, then a keyed random
 * permutation of the positions.
 *
 * Everything is a pure function of (seed, index), so any slice of the output
 * can be produced independently and in parallel:
 *
 *   rng(key, ctr)  = SplitMix64 output function applied to key + (ctr+1)*gamma
 *                    (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *                    generators", OOPSLA 2014).
 *   u01(r)         = (r >> 11) * 2^-53, exact, in [0, 1).
 *   shuffle        = 4-round Feistel network on the smallest even-bit domain
 *                    covering n, restricted to [0, n) by cycle walking
 *                    (Black and Rogaway, "Ciphers with arbitrary finite
 *                    domains", CT-RSA 2002).
 *
 * Position i holds generated point j = perm(i).  Point j < Nc is cluster
 * point number j of cluster (j mod K); points j >= Nc are noise.
 *
 * Only IEEE +, -, * on doubles are used (compile with -ffp-contract=off), so
 * the output is bit-identical on x86-64 and AArch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define GOLDEN_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rng_at(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1u) * GOLDEN_GAMMA);
}

static inline double u01(uint64_t r) {
    return (double)(r >> 11) * 0x1.0p-53;
}

/* Stream keys: one independent stream per purpose. */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed) ^ (stream * 0xd1b54a32d192ed03ULL));
}

enum { ST_CENTRE = 1, ST_OFFSET = 2, ST_NOISE = 3, ST_PERM = 4 };

typedef struct {
    uint64_t n;
    uint64_t half_bits;  /* domain = 2^(2*half_bits) >= n */
    uint64_t mask;       /* (1 << half_bits) - 1 */
    uint64_t rk[4];      /* round keys */
} perm_t;

static void perm_init(perm_t *p, uint64_t n, uint64_t seed) {
    uint64_t hb = 1;
    while (hb < 32 && (1ULL << (2 * hb)) < n) hb++;
    p->n = n;
    p->half_bits = hb;
    p->mask = (1ULL << hb) - 1;
    uint64_t k = stream_key(seed, ST_PERM);
    for (int r = 0; r < 4; ++r) p->rk[r] = rng_at(k, (uint64_t)r);
}

static inline uint64_t feistel(const perm_t *p, uint64_t v) {
    uint64_t l = v >> p->half_bits, r = v & p->mask;
    for (int i = 0; i < 4; ++i) {
        uint64_t nl = r;
        uint64_t nr = l ^ (mix64(r ^ p->rk[i]) & p->mask);
        l = nl;
        r = nr;
    }
    return (l << p->half_bits) | r;
}

static inline uint64_t perm_apply(const perm_t *p, uint64_t i) {
    uint64_t v = feistel(p, i);
    while (v >= p->n) v = feistel(p, v);
    return v;
}

typedef struct {
    double *out;          /* (n, 2) row-major */
    uint64_t lo, hi;      /* positions [lo, hi) */
    uint64_t n, k, nc;
    double canvas, half_width;
    int shuffle;
    perm_t perm;
    uint64_t kc, ko, kn;
} job_t;

static void *run_job(void *arg) {
    job_t *j = (job_t *)arg;
    const double width = 2.0 * j->half_width;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint64_t g = j->shuffle ? perm_apply(&j->perm, i) : i;
        double x, y;
        if (g < j->nc) {
            uint64_t c = g % j->k;
            double cx = u01(rng_at(j->kc, 2 * c)) * j->canvas;
            double cy = u01(rng_at(j->kc, 2 * c + 1)) * j->canvas;
            x = cx + (u01(rng_at(j->ko, 2 * g)) - 0.5) * width;
            y = cy + (u01(rng_at(j->ko, 2 * g + 1)) - 0.5) * width;
        } else {
            x = u01(rng_at(j->kn, 2 * g)) * j->canvas;
            y = u01(rng_at(j->kn, 2 * g + 1)) * j->canvas;
        }
        j->out[2 * i] = x;
        j->out[2 * i + 1] = y;
    }
    return NULL;
}

/*
 * Fill out[lo..hi) (positions) of the workload (n points, k clusters holding
 * nc points in total, canvas L, square half width) for the given seed.
 * out points at position lo.  Returns 0, or -1 on bad arguments.
 */
int gen_points_range(double *out, uint64_t n, uint64_t k, uint64_t nc,
                     double canvas, double half_width, uint64_t seed,
                     int shuffle, uint64_t lo, uint64_t hi, int nthreads) {
    if (!out || hi > n || lo > hi || nc > n || (nc > 0 && k == 0)) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    uint64_t count = hi - lo;
    if ((uint64_t)nthreads > count / 4096 + 1) nthreads = (int)(count / 4096 + 1);
    job_t base;
    base.out = out - 2 * lo;
    base.n = n;
    base.k = k;
    base.nc = nc;
    base.canvas = canvas;
    base.half_width = half_width;
    base.shuffle = shuffle;
    perm_init(&base.perm, n, seed);
    base.kc = stream_key(seed, ST_CENTRE);
    base.ko = stream_key(seed, ST_OFFSET);
    base.kn = stream_key(seed, ST_NOISE);
    job_t jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].lo = lo + count * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = lo + count * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) break;
        started = t;
    }
    run_job(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    /* any job whose thread failed to start runs here */
    for (int t = started + 1; t < nthreads; ++t) run_job(&jobs[t]);
    return 0;
}

/* Counter-based draw, exposed so that per-instance parameters (sizes,
 * precisions) come from the same generator family. */
uint64_t gen_rng_at(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return rng_at(stream_key(seed, stream), ctr);
}

uint64_t gen_perm_apply(uint64_t n, uint64_t seed, uint64_t i) {
    perm_t p;
    perm_init(&p, n, seed);
    return perm_apply(&p, i);
}

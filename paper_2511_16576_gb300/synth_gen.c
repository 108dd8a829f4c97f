/*
 * synth_gen.c -- per-vertex work of the seeded synthetic polygon generator.
 *
 * Input generation only: this file holds none of the hashing method's
 * arithmetic.  synth.py draws the per-polygon parameters (vertex count, area
 * fraction, centre) with numpy and hands the per-vertex work to these
 * routines, which run one polygon at a time on a pool of threads:
 *
 *   sg_star_vertices  vertices of star or fractal-star polygons (before the
 *                     star-shape filter), from a PCG32 generator per polygon;
 *   sg_star_filter    the star-shape filter: drop every vertex v_i with
 *                     (v_i - c) x (v_{i+1} - c) <= 0, repeatedly, until the
 *                     ring turns strictly counter-clockwise around c (a
 *                     polygon left with fewer than 3 vertices becomes a
 *                     triangle around c), in place in each polygon's slot;
 *   sg_compact        packs the kept vertices to the front of the array.
 *
 * The random numbers come from PCG32 (M. E. O'Neill, "PCG: A family of simple
 * fast space-efficient statistically good algorithms for random number
 * generation", 2014: a 64-bit LCG whose output is permuted by an xorshift and
 * a data-dependent rotation), one stream per polygon (stream id = polygon
 * index), so the result does not depend on the number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SG_DOMAIN 65536
#define SG_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* PCG32 (XSH RR), one stream per polygon.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t state, inc;
} pcg32;

static uint32_t pcg32_next(pcg32* g)
{
    const uint64_t old = g->state;
    g->state = old * 6364136223846793005ULL + g->inc;
    const uint32_t xorshifted = (uint32_t)(((old >> 18) ^ old) >> 27);
    const uint32_t rot = (uint32_t)(old >> 59);
    return (xorshifted >> rot) | (xorshifted << ((32u - rot) & 31u));
}

static void pcg32_seed(pcg32* g, uint64_t initstate, uint64_t stream)
{
    g->state = 0;
    g->inc = (stream << 1) | 1u;
    pcg32_next(g);
    g->state += initstate;
    pcg32_next(g);
}

/* uniform double in [0, 1) with 53 random bits */
static double pcg32_unit(pcg32* g)
{
    const uint64_t a = pcg32_next(g) >> 5, b = pcg32_next(g) >> 6;
    return (double)(a * 67108864u + b) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Thread pool over polygon ranges (dynamic chunks of polygons).            */
/* ------------------------------------------------------------------------ */
typedef void (*sg_body)(void* arg, int64_t p, void* scratch);

typedef struct {
    sg_body body;
    void* arg;
    int64_t n, chunk;
    int64_t next;
    pthread_mutex_t lock;
    size_t scratch_bytes;
} sg_pool;

static void* sg_worker(void* vp)
{
    sg_pool* pool = (sg_pool*)vp;
    void* scratch = pool->scratch_bytes ? malloc(pool->scratch_bytes) : NULL;
    for (;;) {
        pthread_mutex_lock(&pool->lock);
        const int64_t a = pool->next;
        pool->next += pool->chunk;
        pthread_mutex_unlock(&pool->lock);
        if (a >= pool->n) break;
        const int64_t b = a + pool->chunk < pool->n ? a + pool->chunk : pool->n;
        for (int64_t p = a; p < b; ++p) pool->body(pool->arg, p, scratch);
    }
    free(scratch);
    return NULL;
}

static void sg_run(sg_body body, void* arg, int64_t n, int nthreads, size_t scratch_bytes)
{
    if (n <= 0) return;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    sg_pool pool;
    pool.body = body;
    pool.arg = arg;
    pool.n = n;
    pool.chunk = n / (nthreads * 64) + 1;
    pool.next = 0;
    pool.scratch_bytes = scratch_bytes;
    pthread_mutex_init(&pool.lock, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, sg_worker, &pool) == 0) ++started;
    sg_worker(&pool);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&pool.lock);
}

/* ------------------------------------------------------------------------ */
/* Star and fractal-star vertices.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int64_t *n, *offs0, *cx, *cy;
    const double* rbar;
    double jitter;
    int fractal;
    uint64_t seed;
    int32_t* xy;
    int64_t max_n;
} star_args;

static int cmp_double(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static int32_t clip_round(double v)
{
    double r = nearbyint(v);
    if (r < 0.0) r = 0.0;
    if (r > (double)SG_DOMAIN) r = (double)SG_DOMAIN;
    return (int32_t)r;
}

/* scratch: max_n angles, max_n radii, 4 * max_n control values */
static void star_body(void* vp, int64_t p, void* scratch)
{
    const star_args* A = (const star_args*)vp;
    const int64_t n = A->n[p];
    double* ang = (double*)scratch;
    double* rad = ang + A->max_n;
    double* ctrl = rad + A->max_n;
    pcg32 g;
    pcg32_seed(&g, A->seed, (uint64_t)p);
    const double rb = A->rbar[p];
    if (A->fractal) {
        /* equally spaced angles with a small jitter; radius = 1 + a periodic
           midpoint-displacement profile: level l adds 2^l control offsets drawn
           in [-amp, amp] (amp = 0.25 * 0.6^(l-2)), interpolated linearly at the
           vertex's position t = i / n; only levels the vertex count resolves
           (2^l <= 2n) and amplitudes >= 1e-4 */
        for (int64_t i = 0; i < n; ++i) {
            ang[i] = ((double)i + 0.1 + 0.8 * pcg32_unit(&g)) * (2.0 * SG_PI) / (double)n;
            rad[i] = 1.0;
        }
        double amp = 0.25;
        for (int lev = 2;; ++lev) {
            const int64_t m = (int64_t)1 << lev;
            if (m > 2 * n || amp < 1e-4) break;
            for (int64_t c = 0; c < m; ++c) ctrl[c] = (2.0 * pcg32_unit(&g) - 1.0) * amp;
            for (int64_t i = 0; i < n; ++i) {
                const double u = (double)i / (double)n * (double)m;
                const double fl = floor(u);
                const int64_t i0 = (int64_t)fl % m, i1 = (i0 + 1) % m;
                const double w = u - fl;
                rad[i] += (1.0 - w) * ctrl[i0] + w * ctrl[i1];
            }
            amp *= 0.6;
        }
        for (int64_t i = 0; i < n; ++i) {
            double r = rad[i];
            r = r < 0.3 ? 0.3 : (r > 1.6 ? 1.6 : r);
            rad[i] = rb * r;
        }
    } else {
        /* sorted uniform angles; a cyclic gap of 0.75 pi or more (which could leave
           the centre outside) switches the polygon to stratified angles */
        for (int64_t i = 0; i < n; ++i) ang[i] = 2.0 * SG_PI * pcg32_unit(&g);
        qsort(ang, (size_t)n, sizeof(double), cmp_double);
        int wide = 0;
        for (int64_t i = 0; i < n; ++i) {
            const double nxt = i + 1 < n ? ang[i + 1] : ang[0] + 2.0 * SG_PI;
            if (nxt - ang[i] > 0.75 * SG_PI) wide = 1;
        }
        if (wide)
            for (int64_t i = 0; i < n; ++i)
                ang[i] = ((double)i + pcg32_unit(&g)) * (2.0 * SG_PI) / (double)n;
        for (int64_t i = 0; i < n; ++i)
            rad[i] = rb * (1.0 - A->jitter + 2.0 * A->jitter * pcg32_unit(&g));
    }
    int32_t* out = A->xy + 2 * A->offs0[p];
    const double cx = (double)A->cx[p], cy = (double)A->cy[p];
    for (int64_t i = 0; i < n; ++i) {
        out[2 * i] = clip_round(cx + rad[i] * cos(ang[i]));
        out[2 * i + 1] = clip_round(cy + rad[i] * sin(ang[i]));
    }
}

void sg_star_vertices(int64_t n_polys, const int64_t* n, const int64_t* offs0, const int64_t* cx,
                      const int64_t* cy, const double* rbar, double jitter, int fractal,
                      uint64_t seed, int nthreads, int32_t* xy)
{
    star_args A = {n, offs0, cx, cy, rbar, jitter, fractal, seed, xy, 1};
    for (int64_t p = 0; p < n_polys; ++p)
        if (n[p] > A.max_n) A.max_n = n[p];
    sg_run(star_body, &A, n_polys, nthreads, sizeof(double) * (size_t)(6 * A.max_n + 8));
}

/* ------------------------------------------------------------------------ */
/* Star-shape filter, in place in each polygon's slot.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int64_t *offs0, *cx, *cy;
    const double* rbar;
    int32_t* xy;
    int64_t* kept;
    int64_t max_n;
} filter_args;

/* scratch: max_n flags */
static void filter_body(void* vp, int64_t p, void* scratch)
{
    const filter_args* A = (const filter_args*)vp;
    int32_t* v = A->xy + 2 * A->offs0[p];
    int64_t n = A->offs0[p + 1] - A->offs0[p];
    unsigned char* bad = (unsigned char*)scratch;
    const int64_t cx = A->cx[p], cy = A->cy[p];
    /* every pass drops all vertices whose edge to the next kept vertex does not
       turn strictly counter-clockwise around c, then checks again */
    for (;;) {
        int64_t nbad = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t j = i + 1 < n ? i + 1 : 0;
            const int64_t ax = (int64_t)v[2 * i] - cx, ay = (int64_t)v[2 * i + 1] - cy;
            const int64_t bx = (int64_t)v[2 * j] - cx, by = (int64_t)v[2 * j + 1] - cy;
            bad[i] = ax * by - bx * ay <= 0;
            nbad += bad[i];
        }
        if (nbad == 0 || n == 0) break;
        int64_t w = 0;
        for (int64_t i = 0; i < n; ++i)
            if (!bad[i]) {
                v[2 * w] = v[2 * i];
                v[2 * w + 1] = v[2 * i + 1];
                ++w;
            }
        n = w;
    }
    if (n < 3) {
        /* a triangle around c of radius max(2, rbar) at angles 0, 2pi/3, 4pi/3 */
        const double r = A->rbar[p] > 2.0 ? A->rbar[p] : 2.0;
        for (int t = 0; t < 3; ++t) {
            const double a = (double)t * 2.0 * SG_PI / 3.0;
            v[2 * t] = (int32_t)nearbyint((double)cx + r * cos(a));
            v[2 * t + 1] = (int32_t)nearbyint((double)cy + r * sin(a));
        }
        n = 3;
    }
    A->kept[p] = n;
}

void sg_star_filter(int64_t n_polys, const int64_t* offs0, int32_t* xy, const int64_t* cx,
                    const int64_t* cy, const double* rbar, int nthreads, int64_t* kept)
{
    filter_args A = {offs0, cx, cy, rbar, xy, kept, 1};
    for (int64_t p = 0; p < n_polys; ++p)
        if (offs0[p + 1] - offs0[p] > A.max_n) A.max_n = offs0[p + 1] - offs0[p];
    sg_run(filter_body, &A, n_polys, nthreads, (size_t)A.max_n + 8);
}

/* ------------------------------------------------------------------------ */
/* Pack the kept vertices to the front of the array, in place (polygon p's   */
/* kept vertices move from offs0[p] to newoffs[p] <= offs0[p], in polygon   */
/* order, so no source is overwritten before it is read).                   */
/* ------------------------------------------------------------------------ */
void sg_compact(int64_t n_polys, const int64_t* offs0, const int64_t* newoffs, int32_t* xy)
{
    for (int64_t p = 0; p < n_polys; ++p)
        if (newoffs[p] != offs0[p])
            memmove(xy + 2 * newoffs[p], xy + 2 * offs0[p],
                    sizeof(int32_t) * 2 * (size_t)(newoffs[p + 1] - newoffs[p]));
}

/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for PolyMinHash.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark; never by the product path.  Shares no code
 * with the CUDA library.
 *
 * Paper: "PolyMinHash: Efficient Area-Based MinHashing of Polygons for
 * Approximate Nearest Neighbor Search" (arXiv 2511.16576).
 *
 * Readings of the paper taken where it is silent or ambiguous:
 *  R1  random points: the paper only asks for seeded uniform sampling over the
 *      global MBR (Sec. 3.2).  Stream k is the SplitMix64 generator (Steele, Lea
 *      & Flood, OOPSLA 2014) seeded with s_k, the (k+1)-th SplitMix64 output of
 *      the global seed; point i is output i+1 of stream k.  The sampling domain
 *      is the integer lattice [0,65536)^2: x = low 16 bits, y = next 16 bits.
 *  R2  membership of a lattice point p is decided for p + (e1, e2) with
 *      0 < e2 << e1 infinitesimal (a half-open rule); the paper only says
 *      "precise point-in-polygon test" (Sec. 3.2, Algorithm 1).
 *  R3  h is 0-based (the number of rejected attempts) and capped at T: if none
 *      of the first T points of stream k lands in P, h = T (Algorithm 1 loops
 *      without bound).
 *  R4  band key: fingerprint of the r-tuple of one band (the paper keys one
 *      hashmap on the whole m-length code, Sec. 3.2 after Thm. 1 and Sec. 5.2).
 *  R5  agreement count: positions where both hashes are equal and not T.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* R1: SplitMix64 (published generator: state += golden gamma, then mix).    */
/* ------------------------------------------------------------------------ */
static const uint64_t GOLDEN_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* s_k: output number k+1 of a SplitMix64 generator whose state starts at seed */
uint64_t orc_stream_seed(uint64_t seed, uint64_t k)
{
    return orc_mix64(seed + (k + 1) * GOLDEN_GAMMA);
}

/* output number i+1 of a SplitMix64 generator whose state starts at s_k */
uint64_t orc_stream_value(uint64_t seed, uint64_t k, uint64_t i)
{
    return orc_mix64(orc_stream_seed(seed, k) + (i + 1) * GOLDEN_GAMMA);
}

/* points i0 .. i0+count-1 of stream k, generated sequentially (state += gamma) */
void orc_stream_points(uint64_t seed, uint64_t k, uint64_t i0, int64_t count,
                       uint32_t* x, uint32_t* y)
{
    uint64_t state = orc_stream_seed(seed, k) + i0 * GOLDEN_GAMMA;
    for (int64_t j = 0; j < count; ++j) {
        state += GOLDEN_GAMMA;
        uint64_t v = orc_mix64(state);
        x[j] = (uint32_t)(v & 0xFFFFu);
        y[j] = (uint32_t)((v >> 16) & 0xFFFFu);
    }
}

/* ------------------------------------------------------------------------ */
/* R2: lattice membership, scanline form.                                    */
/*                                                                          */
/* The point p+(e1,e2) lies on the horizontal line Y = py + e2.  An edge    */
/* a->b meets that line iff min(ay,by) <= py < max(ay,by), at abscissa       */
/* X(py) = ax + (py-ay)(bx-ax)/(by-ay) (up to an e2 term that e1 dominates). */
/* Sorting the crossings c1 <= c2 <= ... of a row, p is inside iff          */
/* c(2m-1) <= px < c(2m) for some m (even-odd rule), and for integer px this */
/* is ceil(c(2m-1)) <= px < ceil(c(2m)).  So each row is a list of integer   */
/* half-open spans.                                                          */
/* ------------------------------------------------------------------------ */
static int64_t ceil_div(int64_t num, int64_t den) /* den > 0 */
{
    int64_t q = num / den;
    if ((num % den) != 0 && num > 0) q += 1;
    return q;
}

typedef struct {
    int64_t y0, y1;      /* rows y0 .. y1-1 */
    int64_t* row_start;  /* [rows+1] index into xs */
    int64_t* xs;         /* sorted span boundaries, pairs [xs[2m], xs[2m+1]) */
} spans_t;

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

static void spans_free(spans_t* s)
{
    free(s->row_start);
    free(s->xs);
    s->row_start = NULL;
    s->xs = NULL;
}

static int spans_build(const int32_t* xy, int64_t n, spans_t* s)
{
    memset(s, 0, sizeof(*s));
    if (n < 1) return 0;
    int64_t ymin = xy[1], ymax = xy[1];
    for (int64_t i = 0; i < n; ++i) {
        if (xy[2 * i + 1] < ymin) ymin = xy[2 * i + 1];
        if (xy[2 * i + 1] > ymax) ymax = xy[2 * i + 1];
    }
    s->y0 = ymin;
    s->y1 = ymax;
    int64_t rows = ymax - ymin;
    s->row_start = (int64_t*)calloc((size_t)rows + 2, sizeof(int64_t));
    if (!s->row_start) return -1;
    /* pass 1: count crossings per row */
    for (int64_t i = 0; i < n; ++i) {
        int64_t ay = xy[2 * i + 1], by = xy[2 * ((i + 1) % n) + 1];
        int64_t lo = ay < by ? ay : by, hi = ay < by ? by : ay;
        for (int64_t y = lo; y < hi; ++y) s->row_start[y - ymin + 1] += 1;
    }
    for (int64_t r = 0; r < rows; ++r) s->row_start[r + 1] += s->row_start[r];
    int64_t total = s->row_start[rows];
    s->xs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    int64_t* fill = (int64_t*)calloc((size_t)rows + 1, sizeof(int64_t));
    if (!s->xs || !fill) {
        free(fill);
        spans_free(s);
        return -1;
    }
    /* pass 2: the ceiling of every crossing abscissa */
    for (int64_t i = 0; i < n; ++i) {
        int64_t ax = xy[2 * i], ay = xy[2 * i + 1];
        int64_t bx = xy[2 * ((i + 1) % n)], by = xy[2 * ((i + 1) % n) + 1];
        if (ay == by) continue;
        int64_t lo = ay < by ? ay : by, hi = ay < by ? by : ay;
        int64_t dx = bx - ax, dy = by - ay;
        for (int64_t y = lo; y < hi; ++y) {
            /* X = ax + (y-ay)*dx/dy = (ax*dy + (y-ay)*dx) / dy */
            int64_t num = ax * dy + (y - ay) * dx, den = dy;
            if (den < 0) {
                num = -num;
                den = -den;
            }
            int64_t r = y - ymin;
            s->xs[s->row_start[r] + fill[r]++] = ceil_div(num, den);
        }
    }
    free(fill);
    for (int64_t r = 0; r < rows; ++r)
        qsort(s->xs + s->row_start[r], (size_t)(s->row_start[r + 1] - s->row_start[r]),
              sizeof(int64_t), cmp_i64);
    return 0;
}

static int spans_contains(const spans_t* s, int64_t px, int64_t py)
{
    if (py < s->y0 || py >= s->y1) return 0;
    int64_t r = py - s->y0;
    for (int64_t j = s->row_start[r]; j + 1 < s->row_start[r + 1]; j += 2)
        if (s->xs[j] <= px && px < s->xs[j + 1]) return 1;
    return 0;
}

/* lattice points of one row inside the domain [0, 65536) */
static int64_t clamp_dom(int64_t v) { return v < 0 ? 0 : (v > 65536 ? 65536 : v); }

int orc_inside(const int32_t* xy, int64_t n, int64_t px, int64_t py)
{
    spans_t s;
    if (spans_build(xy, n, &s) != 0) return -1;
    int r = spans_contains(&s, px, py);
    spans_free(&s);
    return r;
}

/* number of lattice points of [0,65536)^2 inside P */
int64_t orc_lattice_count(const int32_t* xy, int64_t n)
{
    spans_t s;
    if (spans_build(xy, n, &s) != 0) return -1;
    int64_t total = 0;
    for (int64_t y = s.y0; y < s.y1; ++y) {
        if (y < 0 || y >= 65536) continue;
        int64_t r = y - s.y0;
        for (int64_t j = s.row_start[r]; j + 1 < s.row_start[r + 1]; j += 2)
            total += clamp_dom(s.xs[j + 1]) - clamp_dom(s.xs[j]);
    }
    spans_free(&s);
    return total;
}

/* lattice counts of A, B and A n B (row spans intersected exactly) */
int orc_lattice_pair(const int32_t* a, int64_t na, const int32_t* b, int64_t nb,
                     int64_t* count_a, int64_t* count_b, int64_t* count_ab)
{
    spans_t sa, sb;
    if (spans_build(a, na, &sa) != 0) return -1;
    if (spans_build(b, nb, &sb) != 0) {
        spans_free(&sa);
        return -1;
    }
    *count_a = orc_lattice_count(a, na);
    *count_b = orc_lattice_count(b, nb);
    int64_t both = 0;
    int64_t ylo = sa.y0 > sb.y0 ? sa.y0 : sb.y0, yhi = sa.y1 < sb.y1 ? sa.y1 : sb.y1;
    for (int64_t y = ylo; y < yhi; ++y) {
        if (y < 0 || y >= 65536) continue;
        int64_t ra = y - sa.y0, rb = y - sb.y0;
        for (int64_t i = sa.row_start[ra]; i + 1 < sa.row_start[ra + 1]; i += 2)
            for (int64_t j = sb.row_start[rb]; j + 1 < sb.row_start[rb + 1]; j += 2) {
                int64_t lo = sa.xs[i] > sb.xs[j] ? sa.xs[i] : sb.xs[j];
                int64_t hi = sa.xs[i + 1] < sb.xs[j + 1] ? sa.xs[i + 1] : sb.xs[j + 1];
                lo = clamp_dom(lo);
                hi = clamp_dom(hi);
                if (hi > lo) both += hi - lo;
            }
    }
    *count_ab = both;
    spans_free(&sa);
    spans_free(&sb);
    return 0;
}

/* twice the signed area, shoelace formula, exact in int64 */
int64_t orc_area2(const int32_t* xy, int64_t n)
{
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = (i + 1) % n;
        s += (int64_t)xy[2 * i] * xy[2 * j + 1] - (int64_t)xy[2 * j] * xy[2 * i + 1];
    }
    return s;
}

/* local MBR of P (Sec. 3.1): xmin, ymin, xmax, ymax */
void orc_bbox(const int32_t* xy, int64_t n, int32_t* bbox4)
{
    int32_t x0 = xy[0], y0 = xy[1], x1 = xy[0], y1 = xy[1];
    for (int64_t i = 1; i < n; ++i) {
        if (xy[2 * i] < x0) x0 = xy[2 * i];
        if (xy[2 * i] > x1) x1 = xy[2 * i];
        if (xy[2 * i + 1] < y0) y0 = xy[2 * i + 1];
        if (xy[2 * i + 1] > y1) y1 = xy[2 * i + 1];
    }
    bbox4[0] = x0;
    bbox4[1] = y0;
    bbox4[2] = x1;
    bbox4[3] = y1;
}

/* ------------------------------------------------------------------------ */
/* Definition 2 with R1-R3: h_k(P) = min{ i in [0,T) : point(k,i) in P },    */
/* else T.  The walk follows Algorithm 1: draw a point, reject it if it is  */
/* outside the local MBR, else run the exact membership test.  A polygon    */
/* that holds no lattice point of the domain can never be hit, so its       */
/* hashes are T without walking the stream (same result, exactly).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int32_t* xy;
    const int64_t* offsets;
    int64_t p0, p1;
    uint64_t seed;
    uint32_t K, T;
    uint32_t* hashes;
    int64_t *points, *bbox_hits, *edge_tests;
    int status;
} sign_job_t;

static void* sign_range(void* arg)
{
    sign_job_t* job = (sign_job_t*)arg;
    for (int64_t p = job->p0; p < job->p1; ++p) {
        const int32_t* v = job->xy + 2 * job->offsets[p];
        int64_t n = job->offsets[p + 1] - job->offsets[p];
        int64_t pts = 0, hits = 0;
        uint32_t* h = job->hashes + (size_t)p * job->K;
        spans_t s;
        if (n < 3 || spans_build(v, n, &s) != 0) {
            job->status = -1;
            return NULL;
        }
        int32_t bb[4];
        orc_bbox(v, n, bb);
        int64_t lattice = orc_lattice_count(v, n);
        for (uint32_t k = 0; k < job->K; ++k) {
            h[k] = job->T;
            if (lattice == 0) continue;
            uint64_t state = orc_stream_seed(job->seed, k);
            for (uint32_t i = 0; i < job->T; ++i) {
                state += GOLDEN_GAMMA;
                uint64_t z = orc_mix64(state);
                int64_t x = (int64_t)(z & 0xFFFFu), y = (int64_t)((z >> 16) & 0xFFFFu);
                ++pts;
                if (x < bb[0] || x >= bb[2] || y < bb[1] || y >= bb[3]) continue;
                ++hits;
                if (spans_contains(&s, x, y)) {
                    h[k] = i;
                    break;
                }
            }
        }
        spans_free(&s);
        if (job->points) job->points[p] = pts;
        if (job->bbox_hits) job->bbox_hits[p] = hits;
        if (job->edge_tests) job->edge_tests[p] = hits * n;
    }
    return NULL;
}

int orc_sign(const int32_t* xy, const int64_t* offsets, int64_t n_polys, uint64_t seed,
             uint32_t K, uint32_t T, uint32_t* hashes, int nthreads)
{
    enum { MAX_THREADS = 512 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAX_THREADS) nthreads = MAX_THREADS;
    sign_job_t jobs[MAX_THREADS];
    pthread_t tid[MAX_THREADS];
    int joined[MAX_THREADS];
    int64_t per = (n_polys + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        int64_t p0 = (int64_t)t * per, p1 = (int64_t)(t + 1) * per;
        sign_job_t j = {xy, offsets, p0 < n_polys ? p0 : n_polys, p1 < n_polys ? p1 : n_polys,
                        seed, K, T, hashes, NULL, NULL, NULL, 0};
        jobs[t] = j;
        joined[t] = 0;
    }
    for (int t = 0; t < nthreads; ++t) {
        if (nthreads > 1 && pthread_create(&tid[t], NULL, sign_range, &jobs[t]) == 0)
            joined[t] = 1;
        else
            sign_range(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (joined[t]) pthread_join(tid[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status != 0) return -1;
    return 0;
}

/* the same walk, single-threaded, also reporting the work it did per polygon */
int orc_sign_work(const int32_t* xy, const int64_t* offsets, int64_t n_polys, uint64_t seed,
                  uint32_t K, uint32_t T, uint32_t* hashes, int64_t* points,
                  int64_t* bbox_hits, int64_t* edge_tests)
{
    sign_job_t j = {xy, offsets, 0, n_polys, seed, K, T, hashes,
                    points, bbox_hits, edge_tests, 0};
    sign_range(&j);
    return j.status;
}

/* ------------------------------------------------------------------------ */
/* R4: band keys.  Band j covers hashes j*r .. j*r+r-1.                       */
/*   a = mix64(lsh_seed + (j+1)*gamma); a = mix64(a ^ h) for each row h;    */
/*   key = a (the all-ones value is moved to all-ones minus one);           */
/*   a band holding the sentinel T has the invalid key (all ones).          */
/* ------------------------------------------------------------------------ */
void orc_band_keys(const uint32_t* hashes, int64_t n, uint32_t K, uint32_t bands,
                   uint32_t rows, uint32_t T, uint64_t lsh_seed, uint64_t* keys)
{
    for (int64_t p = 0; p < n; ++p)
        for (uint32_t j = 0; j < bands; ++j) {
            uint64_t a = orc_mix64(lsh_seed + (uint64_t)(j + 1) * GOLDEN_GAMMA);
            int valid = 1;
            for (uint32_t t = 0; t < rows; ++t) {
                uint32_t h = hashes[(size_t)p * K + (size_t)j * rows + t];
                if (h == T) valid = 0;
                a = orc_mix64(a ^ (uint64_t)h);
            }
            if (a == ~0ULL) a = ~0ULL - 1;
            keys[(size_t)p * bands + j] = valid ? a : ~0ULL;
        }
}

/* ------------------------------------------------------------------------ */
/* Candidate set of query q (hashmap buckets, one map per band):             */
/*   C(q) = { p : some band j has a valid r-tuple in both and equal tuples } */
/* Written as the O(Q*N*b) definition; ids ascending, no duplicates.        */
/* Returns the total number of candidates; fills cand only up to cap.       */
/* ------------------------------------------------------------------------ */
static int band_tuple_equal(const uint32_t* a, const uint32_t* b, uint32_t j, uint32_t rows,
                            uint32_t T)
{
    for (uint32_t t = 0; t < rows; ++t) {
        uint32_t x = a[j * rows + t], y = b[j * rows + t];
        if (x == T || y == T || x != y) return 0;
    }
    return 1;
}

int64_t orc_candidates(const uint32_t* qh, int64_t Q, const uint32_t* ph, int64_t N,
                       uint32_t K, uint32_t bands, uint32_t rows, uint32_t T,
                       int64_t* row_ptr, int32_t* cand, int64_t cap)
{
    int64_t total = 0;
    row_ptr[0] = 0;
    for (int64_t q = 0; q < Q; ++q) {
        const uint32_t* a = qh + (size_t)q * K;
        for (int64_t p = 0; p < N; ++p) {
            const uint32_t* b = ph + (size_t)p * K;
            int hit = 0;
            for (uint32_t j = 0; j < bands && !hit; ++j) hit = band_tuple_equal(a, b, j, rows, T);
            if (hit) {
                if (total < cap) cand[total] = (int32_t)p;
                ++total;
            }
        }
        row_ptr[q + 1] = total;
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Theorem 1: Pr[h_k(q) = h_k(p)] = J(q,p).  Count of agreeing positions    */
/* (R5: the sentinel T never agrees) and the per-band full-match bits.      */
/* ------------------------------------------------------------------------ */
void orc_agree(const uint32_t* qh, const uint32_t* ph, uint32_t K, uint32_t bands,
               uint32_t rows, uint32_t T, const int64_t* row_ptr, const int32_t* cand,
               int64_t Q, uint16_t* count, uint32_t* bandmask)
{
    for (int64_t q = 0; q < Q; ++q)
        for (int64_t e = row_ptr[q]; e < row_ptr[q + 1]; ++e) {
            const uint32_t* a = qh + (size_t)q * K;
            const uint32_t* b = ph + (size_t)cand[e] * K;
            uint32_t c = 0;
            for (uint32_t k = 0; k < K; ++k) c += (a[k] == b[k] && a[k] != T);
            count[e] = (uint16_t)c;
            if (bandmask) {
                uint32_t m = 0;
                for (uint32_t j = 0; j < bands && j < 32; ++j)
                    if (band_tuple_equal(a, b, j, rows, T)) m |= 1u << j;
                bandmask[e] = m;
            }
        }
}

/* top-m of every candidate row by (count descending, id ascending) */
typedef struct {
    int32_t id;
    uint16_t c;
} cid_t;

static int cmp_cid(const void* a, const void* b)
{
    const cid_t* x = (const cid_t*)a;
    const cid_t* y = (const cid_t*)b;
    if (x->c != y->c) return x->c > y->c ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

int orc_topm_by_count(const int64_t* row_ptr, const int32_t* cand, const uint16_t* count,
                      int64_t Q, int32_t m, int32_t* out_ids, int32_t* out_n)
{
    for (int64_t q = 0; q < Q; ++q) {
        int64_t n = row_ptr[q + 1] - row_ptr[q];
        cid_t* tmp = (cid_t*)malloc(sizeof(cid_t) * (size_t)(n > 0 ? n : 1));
        if (!tmp) return -1;
        for (int64_t e = 0; e < n; ++e) {
            tmp[e].id = cand[row_ptr[q] + e];
            tmp[e].c = count[row_ptr[q] + e];
        }
        qsort(tmp, (size_t)n, sizeof(cid_t), cmp_cid);
        int32_t keep = n < m ? (int32_t)n : m;
        for (int32_t e = 0; e < m; ++e) out_ids[q * m + e] = e < keep ? tmp[e].id : -1;
        out_n[q] = keep;
        free(tmp);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact Jaccard J = area(A n B) / area(A u B) (Sec. 1).                     */
/*                                                                          */
/* Intersection area by a horizontal slab sweep: cut the plane at every      */
/* vertex y of A and B and at the y of every point where an edge of A meets  */
/* an edge of B.  Inside one slab no two edges cross and no vertex lies, so  */
/* the even-odd intervals of A and of B at height y have endpoints that are  */
/* linear in y, in a fixed order, and the length of their intersection is    */
/* linear in y: the slab contributes height * length(mid-height).           */
/* area(A u B) = area(A) + area(B) - area(A n B), areas by the shoelace.     */
/* ------------------------------------------------------------------------ */
static int cmp_ld(const void* a, const void* b)
{
    long double x = *(const long double*)a, y = *(const long double*)b;
    return (x > y) - (x < y);
}

/* sorted crossing abscissae of the line Y = y with the edges of P */
static int64_t row_crossings(const int32_t* p, int64_t n, long double y, long double* out)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        long double ax = p[2 * i], ay = p[2 * i + 1];
        long double bx = p[2 * ((i + 1) % n)], by = p[2 * ((i + 1) % n) + 1];
        if ((ay <= y && y < by) || (by <= y && y < ay))
            out[c++] = ax + (y - ay) * (bx - ax) / (by - ay);
    }
    qsort(out, (size_t)c, sizeof(long double), cmp_ld);
    return c;
}

static int64_t orient_sign(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy)
{
    __int128 v = (__int128)(bx - ax) * (cy - ay) - (__int128)(by - ay) * (cx - ax);
    return (v > 0) - (v < 0);
}

double orc_intersection_area(const int32_t* a, int64_t na, const int32_t* b, int64_t nb)
{
    int64_t cap = na + nb + 4 * na * nb + 4;
    long double* ys = (long double*)malloc(sizeof(long double) * (size_t)cap);
    long double* ca = (long double*)malloc(sizeof(long double) * (size_t)(na + 1));
    long double* cb = (long double*)malloc(sizeof(long double) * (size_t)(nb + 1));
    if (!ys || !ca || !cb) {
        free(ys);
        free(ca);
        free(cb);
        return -1.0;
    }
    int64_t ny = 0;
    for (int64_t i = 0; i < na; ++i) ys[ny++] = a[2 * i + 1];
    for (int64_t i = 0; i < nb; ++i) ys[ny++] = b[2 * i + 1];
    for (int64_t i = 0; i < na; ++i) {
        int64_t p0x = a[2 * i], p0y = a[2 * i + 1];
        int64_t p1x = a[2 * ((i + 1) % na)], p1y = a[2 * ((i + 1) % na) + 1];
        for (int64_t j = 0; j < nb; ++j) {
            int64_t q0x = b[2 * j], q0y = b[2 * j + 1];
            int64_t q1x = b[2 * ((j + 1) % nb)], q1y = b[2 * ((j + 1) % nb) + 1];
            int64_t o1 = orient_sign(p0x, p0y, p1x, p1y, q0x, q0y);
            int64_t o2 = orient_sign(p0x, p0y, p1x, p1y, q1x, q1y);
            int64_t o3 = orient_sign(q0x, q0y, q1x, q1y, p0x, p0y);
            int64_t o4 = orient_sign(q0x, q0y, q1x, q1y, p1x, p1y);
            if (o1 * o2 > 0 || o3 * o4 > 0) continue;        /* no contact */
            if (o1 == 0 && o2 == 0) continue;                /* collinear: endpoints are vertices */
            /* one contact point: solve p0 + t (p1-p0) on the line through q */
            long double dx = (long double)(p1x - p0x), dy = (long double)(p1y - p0y);
            long double ex = (long double)(q1x - q0x), ey = (long double)(q1y - q0y);
            long double den = dx * ey - dy * ex;
            if (den == 0) continue;
            long double t = ((long double)(q0x - p0x) * ey - (long double)(q0y - p0y) * ex) / den;
            ys[ny++] = (long double)p0y + t * dy;
        }
    }
    qsort(ys, (size_t)ny, sizeof(long double), cmp_ld);
    long double area = 0;
    for (int64_t s = 0; s + 1 < ny; ++s) {
        long double h = ys[s + 1] - ys[s];
        if (!(h > 0)) continue;
        long double ym = 0.5L * (ys[s] + ys[s + 1]);
        int64_t nca = row_crossings(a, na, ym, ca);
        int64_t ncb = row_crossings(b, nb, ym, cb);
        long double len = 0;
        for (int64_t i = 0; i + 1 < nca; i += 2)
            for (int64_t j = 0; j + 1 < ncb; j += 2) {
                long double lo = ca[i] > cb[j] ? ca[i] : cb[j];
                long double hi = ca[i + 1] < cb[j + 1] ? ca[i + 1] : cb[j + 1];
                if (hi > lo) len += hi - lo;
            }
        area += h * len;
    }
    free(ys);
    free(ca);
    free(cb);
    return (double)area;
}

double orc_jaccard(const int32_t* a, int64_t na, const int32_t* b, int64_t nb)
{
    double inter = orc_intersection_area(a, na, b, nb);
    double aa = fabs((double)orc_area2(a, na)) * 0.5;
    double ab = fabs((double)orc_area2(b, nb)) * 0.5;
    double uni = aa + ab - inter;
    if (!(uni > 0)) return 0.0;
    return inter / uni;
}

/* ------------------------------------------------------------------------ */
/* Reranker MLP reference: 3 layers d_in -> d_h -> d_h -> 1, ReLU, ReLU,     */
/* sigmoid, mean squared error on the label.  Every GEMM operand (weights,  */
/* layer inputs, back-propagated gradients) is rounded to bf16              */
/* (round-to-nearest-even) when emulate_bf16 is set; sums are exact fp64    */
/* (the GPU accumulates fp32).  With emulate_bf16 = 0 it is the exact fp64  */
/* network, which finite differences pin.                                   */
/* Weight layout: w1 [d_h][d_in], w2 [d_h][d_h], w3 [d_h], row-major        */
/* (out, in).  Gradients are of the loss w.r.t. the master weights.         */
/* ------------------------------------------------------------------------ */
double orc_bf16_round(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (double)f; /* inf / nan */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* a GEMM operand: rounded to bf16 when the bf16 network is emulated */
static double operand(int emulate_bf16, double v)
{
    return emulate_bf16 ? orc_bf16_round(v) : v;
}

void orc_mlp_forward_backward(const float* x, const float* y, int64_t n_rows, int32_t d_in,
                              int32_t d_h, const double* w1, const double* b1,
                              const double* w2, const double* b2, const double* w3,
                              const double* b3, double* pred, double* loss, double* gw1,
                              double* gb1, double* gw2, double* gb2, double* gw3, double* gb3,
                              int emulate_bf16)
{
    double* z1 = (double*)calloc((size_t)d_h, sizeof(double));
    double* h1 = (double*)calloc((size_t)d_h, sizeof(double));
    double* z2 = (double*)calloc((size_t)d_h, sizeof(double));
    double* h2 = (double*)calloc((size_t)d_h, sizeof(double));
    double* d2 = (double*)calloc((size_t)d_h, sizeof(double));
    double* d1 = (double*)calloc((size_t)d_h, sizeof(double));
    double* xin = (double*)calloc((size_t)d_in, sizeof(double));
    if (gw1) memset(gw1, 0, sizeof(double) * (size_t)d_h * d_in);
    if (gb1) memset(gb1, 0, sizeof(double) * (size_t)d_h);
    if (gw2) memset(gw2, 0, sizeof(double) * (size_t)d_h * d_h);
    if (gb2) memset(gb2, 0, sizeof(double) * (size_t)d_h);
    if (gw3) memset(gw3, 0, sizeof(double) * (size_t)d_h);
    if (gb3) *gb3 = 0;
    double L = 0;
    for (int64_t r = 0; r < n_rows; ++r) {
        for (int32_t i = 0; i < d_in; ++i) xin[i] = operand(emulate_bf16, x[r * d_in + i]);
        for (int32_t o = 0; o < d_h; ++o) {
            double s = b1[o];
            for (int32_t i = 0; i < d_in; ++i) s += operand(emulate_bf16, w1[o * d_in + i]) * xin[i];
            z1[o] = s;
            h1[o] = operand(emulate_bf16, s > 0 ? s : 0);
        }
        for (int32_t o = 0; o < d_h; ++o) {
            double s = b2[o];
            for (int32_t i = 0; i < d_h; ++i) s += operand(emulate_bf16, w2[o * d_h + i]) * h1[i];
            z2[o] = s;
            h2[o] = operand(emulate_bf16, s > 0 ? s : 0);
        }
        double z3 = b3[0];
        for (int32_t i = 0; i < d_h; ++i) z3 += operand(emulate_bf16, w3[i]) * h2[i];
        double p = 1.0 / (1.0 + exp(-z3));
        pred[r] = p;
        double err = p - (double)y[r];
        L += err * err;
        if (!gw1) continue;
        /* dL/dz3 for L = mean (p - y)^2 */
        double g3 = 2.0 * err / (double)n_rows * p * (1.0 - p);
        double g3r = operand(emulate_bf16, g3);
        for (int32_t i = 0; i < d_h; ++i) gw3[i] += g3r * h2[i];
        *gb3 += g3;
        for (int32_t i = 0; i < d_h; ++i) {
            double dh = operand(emulate_bf16, w3[i]) * g3r;
            d2[i] = operand(emulate_bf16, z2[i] > 0 ? dh : 0);
        }
        for (int32_t o = 0; o < d_h; ++o) {
            gb2[o] += z2[o] > 0 ? operand(emulate_bf16, w3[o]) * g3r : 0;
            for (int32_t i = 0; i < d_h; ++i) gw2[o * d_h + i] += d2[o] * h1[i];
        }
        for (int32_t i = 0; i < d_h; ++i) {
            double dh = 0;
            for (int32_t o = 0; o < d_h; ++o) dh += operand(emulate_bf16, w2[o * d_h + i]) * d2[o];
            d1[i] = z1[i] > 0 ? dh : 0;
        }
        for (int32_t o = 0; o < d_h; ++o) {
            gb1[o] += d1[o];
            double d1r = operand(emulate_bf16, d1[o]);
            for (int32_t i = 0; i < d_in; ++i) gw1[o * d_in + i] += d1r * xin[i];
        }
    }
    *loss = L / (double)(n_rows > 0 ? n_rows : 1);
    free(z1);
    free(h1);
    free(z2);
    free(h2);
    free(d2);
    free(d1);
    free(xin);
}

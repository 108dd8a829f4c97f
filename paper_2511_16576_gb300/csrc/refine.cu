// refine.cu -- step A8: exact Jaccard refinement (Sec. 5.2 refinement phase;
// J = area(A n B) / area(A u B), Sec. 1).
//
// area(A n B) by Green's theorem: the boundary of A n B is made of the pieces
// of A's edges inside B and of B's edges inside A, and area = closed integral
// of x dy over it.  Along one edge the pieces need not be sorted: with
// F(t) = dy * (x0 t + dx t^2 / 2) (x dy integrated from the edge start to
// parameter t), an edge that starts inside contributes nothing at t = 0, every
// crossing where it enters the other polygon contributes -F(t), every exit
// +F(t), and an edge that ends inside adds F(1).  So each (edge, edge) pair is
// independent and a block sums them in any order.
//
// Degenerate contacts (a vertex on an edge, overlapping collinear edges,
// identical polygons) are resolved by simulation of simplicity: A is taken as
// shifted by (e1, e2), 0 < e2 << e1 infinitesimal.  Every predicate is then
// decided exactly with int64 cross products (coordinates <= 2^20), and the
// area of the shifted configuration tends to the exact one.  Crossing
// parameters and the integrals are fp64 in coordinates relative to B's first
// vertex.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kRefineThreads = 128;
constexpr int kSmemVerts = 4096;  // both polygons staged when n_a + n_b fits

__device__ __forceinline__ long long cross3(int2 o, int2 a, int2 b)
{
    return (long long)(a.x - o.x) * (b.y - o.y) - (long long)(a.y - o.y) * (b.x - o.x);
}

// sign of orient(c, d, p + e)
__device__ __forceinline__ int side_of_shifted_point(int2 c, int2 d, int2 p)
{
    long long o = cross3(c, d, p);
    if (o != 0) return o > 0 ? 1 : -1;
    int dy = d.y - c.y, dx = d.x - c.x;
    if (dy != 0) return dy > 0 ? -1 : 1;
    return dx > 0 ? 1 : -1;
}

// sign of orient(a + e, b + e, q)
__device__ __forceinline__ int side_of_point_to_shifted(int2 a, int2 b, int2 q)
{
    long long o = cross3(a, b, q);
    if (o != 0) return o > 0 ? 1 : -1;
    int dy = b.y - a.y, dx = b.x - a.x;
    if (dy != 0) return dy > 0 ? 1 : -1;
    return dx > 0 ? -1 : 1;
}

__device__ __forceinline__ double Fint(double x0, double dx, double dy, double t)
{
    return dy * (x0 * t + 0.5 * dx * t * t);
}

__device__ __forceinline__ bool boxes_touch(int2 a, int2 b, int2 c, int2 d)
{
    return max(min(a.x, b.x), min(c.x, d.x)) <= min(max(a.x, b.x), max(c.x, d.x)) &&
           max(min(a.y, b.y), min(c.y, d.y)) <= min(max(a.y, b.y), max(c.y, d.y));
}

__device__ double block_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

// area(A n B) for one pair, by the whole block; valid in thread 0
__device__ double intersection_area(const int2* __restrict__ A, int na, int sA,
                                    const int2* __restrict__ B, int nb, int sB, double* sh)
{
    const int2 org = B[0];
    double acc = 0;
    // pieces of A's (shifted) edges inside B
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        int2 a = A[i], b = A[i + 1 == na ? 0 : i + 1];
        if (a.x == b.x && a.y == b.y) continue;
        double x0 = (double)(a.x - org.x), dx = (double)(b.x - a.x), dy = (double)(b.y - a.y);
        unsigned start_in = 0, ncross = 0;
        double s = 0;
        for (int j = 0; j < nb; ++j) {
            int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
            // a + e inside B: half-open crossing rule for the point a
            if ((c.y > a.y) != (d.y > a.y)) {
                long long cr = cross3(c, d, a);
                start_in ^= (cr != 0) & ((cr > 0) == (d.y > c.y));
            }
            if (!boxes_touch(a, b, c, d) || (c.x == d.x && c.y == d.y)) continue;
            int s1 = side_of_shifted_point(c, d, a), s2 = side_of_shifted_point(c, d, b);
            if (s1 == s2) continue;
            int s3 = side_of_point_to_shifted(a, b, c), s4 = side_of_point_to_shifted(a, b, d);
            if (s3 == s4) continue;
            double ex = (double)(d.x - c.x), ey = (double)(d.y - c.y);
            double den = dx * ey - dy * ex;
            double t = ((double)(c.x - a.x) * ey - (double)(c.y - a.y) * ex) / den;
            t = fmin(fmax(t, 0.0), 1.0);
            bool entering = (s2 > 0) == (sB > 0);
            double f = Fint(x0, dx, dy, t);
            s += entering ? -f : f;
            ++ncross;
        }
        if ((start_in ^ (ncross & 1u)) != 0) s += Fint(x0, dx, dy, 1.0);
        acc += sA > 0 ? s : -s;
    }
    // pieces of B's edges inside the shifted A
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
        if (c.x == d.x && c.y == d.y) continue;
        double x0 = (double)(c.x - org.x), ex = (double)(d.x - c.x), ey = (double)(d.y - c.y);
        unsigned start_in = 0, ncross = 0;
        double s = 0;
        for (int i = 0; i < na; ++i) {
            int2 a = A[i], b = A[i + 1 == na ? 0 : i + 1];
            // c - e inside A
            if ((a.y >= c.y) != (b.y >= c.y)) {
                long long cr = cross3(a, b, c);
                start_in ^= (cr == 0) | ((cr > 0) == (b.y > a.y));
            }
            if (!boxes_touch(a, b, c, d) || (a.x == b.x && a.y == b.y)) continue;
            int s1 = side_of_shifted_point(c, d, a), s2 = side_of_shifted_point(c, d, b);
            if (s1 == s2) continue;
            int s3 = side_of_point_to_shifted(a, b, c), s4 = side_of_point_to_shifted(a, b, d);
            if (s3 == s4) continue;
            double dx = (double)(b.x - a.x), dy = (double)(b.y - a.y);
            double den = dx * ey - dy * ex;
            double u = ((double)(c.x - a.x) * dy - (double)(c.y - a.y) * dx) / den;
            u = fmin(fmax(u, 0.0), 1.0);
            bool entering = (s4 > 0) == (sA > 0);
            double f = Fint(x0, ex, ey, u);
            s += entering ? -f : f;
            ++ncross;
        }
        if ((start_in ^ (ncross & 1u)) != 0) s += Fint(x0, ex, ey, 1.0);
        acc += sB > 0 ? s : -s;
    }
    return block_sum(acc, sh);
}

struct PairView {
    const int2* v;
    int n;
    int sgn;
    double area;
};

__device__ __forceinline__ PairView view(const int2* xy, const int64_t* off, const int64_t* area2,
                                         int64_t p)
{
    PairView r;
    int64_t b = off[p];
    r.v = xy + b;
    r.n = (int)(off[p + 1] - b);
    long long a2 = area2[p];
    r.sgn = a2 > 0 ? 1 : (a2 < 0 ? -1 : 0);
    r.area = 0.5 * fabs((double)a2);
    return r;
}

// stage both polygons in shared memory when they fit, then compute J
__device__ double pair_jaccard(PairView A, PairView B, int2* sv, double* sh)
{
    if (A.sgn == 0 || B.sgn == 0) return 0.0;
    const int2* a = A.v;
    const int2* b = B.v;
    if (A.n + B.n <= kSmemVerts) {
        for (int i = threadIdx.x; i < A.n; i += blockDim.x) sv[i] = A.v[i];
        for (int i = threadIdx.x; i < B.n; i += blockDim.x) sv[A.n + i] = B.v[i];
        __syncthreads();
        a = sv;
        b = sv + A.n;
    }
    double inter = intersection_area(a, A.n, A.sgn, b, B.n, B.sgn, sh);
    __syncthreads();
    double uni = A.area + B.area - inter;
    return uni > 0 ? fmin(fmax(inter / uni, 0.0), 1.0) : 0.0;
}

__global__ void __launch_bounds__(kRefineThreads)
refine_pairs_kernel(const int2* __restrict__ qxy, const int64_t* __restrict__ qoff,
                    const int64_t* __restrict__ qarea2, const int2* __restrict__ pxy,
                    const int64_t* __restrict__ poff, const int64_t* __restrict__ parea2,
                    const int32_t* __restrict__ ids, const int32_t* __restrict__ nlist, int m,
                    const int32_t* __restrict__ qid_list, int64_t n_pairs, double* __restrict__ out)
{
    __shared__ int2 sv[kSmemVerts];
    __shared__ double sh[kRefineThreads / 32];
    for (int64_t e = blockIdx.x; e < n_pairs; e += gridDim.x) {
        int64_t q;
        int32_t p;
        if (qid_list) {  // explicit pairs
            q = qid_list[e];
            p = ids[e];
        } else {         // top-m lists: pair e = (q, slot)
            q = e / m;
            int slot = (int)(e - q * m);
            if (slot >= nlist[q]) {
                if (threadIdx.x == 0) out[e] = -1.0;
                continue;
            }
            p = ids[e];
        }
        double j = pair_jaccard(view(qxy, qoff, qarea2, q), view(pxy, poff, parea2, p), sv, sh);
        if (threadIdx.x == 0) out[e] = j;
        __syncthreads();
    }
}

struct JKey {
    double j;
    int32_t id;
};

__device__ __forceinline__ bool jkey_before(JKey a, JKey b)  // (J desc, id asc)
{
    return a.j > b.j || (a.j == b.j && (uint32_t)a.id < (uint32_t)b.id);
}

__global__ void topk_by_j_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ nlist,
                                 const double* __restrict__ jv, int m, int cap, int k,
                                 int32_t* __restrict__ top_ids, double* __restrict__ top_j)
{
    extern __shared__ JKey s[];
    const int64_t q = blockIdx.x;
    const int n = nlist[q];
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        JKey x;
        if (i < n) {
            x.j = jv[q * m + i];
            x.id = ids[q * m + i];
        } else {
            x.j = -1.0;
            x.id = -1;  // as unsigned: largest id, sorts last
        }
        s[i] = x;
    }
    __syncthreads();
    for (int kk = 2; kk <= cap; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < cap; i += blockDim.x) {
                int l = i ^ jj;
                if (l > i) {
                    JKey a = s[i], b = s[l];
                    bool up = (i & kk) == 0;
                    if (jkey_before(b, a) == up) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        bool ok = i < n;
        top_ids[q * k + i] = ok ? s[i].id : -1;
        top_j[q * k + i] = ok ? s[i].j : -1.0;
    }
}

}  // namespace

extern "C" int pmh_refine_topk(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_ids,
                               const int32_t* d_n, int64_t Q, int32_t m, int32_t k,
                               int32_t* d_top_ids, double* d_top_j, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!queries || !db || Q < 0 || Q > queries->n || m < 1 || m > 1024 || k < 1 || k > m ||
        (Q > 0 && (!d_ids || !d_n || !d_top_ids || !d_top_j)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (1 <= k <= m <= 1024)");
    if (Q == 0) return PMH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double* jv = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_REFINE, sizeof(double) * (size_t)(Q * m), (void**)&jv));
    int64_t n_pairs = Q * m;
    int blocks = (int)std::min<int64_t>(n_pairs, (int64_t)ctx->sm_count * 16);
    refine_pairs_kernel<<<blocks, kRefineThreads, 0, s>>>(
        queries->xy, queries->offsets, queries->area2, db->xy, db->offsets, db->area2, d_ids, d_n, m,
        nullptr, n_pairs, jv);
    PMH_LAUNCHED("refine_pairs_kernel");
    int cap = 1;
    while (cap < m) cap <<= 1;
    size_t smem = sizeof(JKey) * cap;
    topk_by_j_kernel<<<(unsigned)Q, 256, smem, s>>>(d_ids, d_n, jv, m, cap, k, d_top_ids, d_top_j);
    PMH_LAUNCHED("topk_by_j_kernel");
    return PMH_OK;
}

extern "C" int pmh_pair_jaccard(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_qid,
                                const int32_t* d_pid, int64_t n_pairs, double* d_j, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!queries || !db || n_pairs < 0 || (n_pairs > 0 && (!d_qid || !d_pid || !d_j)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    if (n_pairs == 0) return PMH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int blocks = (int)std::min<int64_t>(n_pairs, (int64_t)ctx->sm_count * 16);
    refine_pairs_kernel<<<blocks, kRefineThreads, 0, s>>>(
        queries->xy, queries->offsets, queries->area2, db->xy, db->offsets, db->area2, d_pid,
        nullptr, 1, d_qid, n_pairs, d_j);
    PMH_LAUNCHED("refine_pairs_kernel");
    return PMH_OK;
}

// ---------------------------------------------------------------------------
// Brute-force candidate set of the exact search (the paper's BF baseline,
// Sec. 5.2): every database polygon whose bounding box overlaps the query's
// with positive area -- the only ones with J > 0.  One warp per query scans
// the database 32 polygons at a time; ballots keep ids ascending.
// ---------------------------------------------------------------------------
namespace {

template <bool kWrite>
__global__ void bbox_join_kernel(const int4* __restrict__ qbox, int64_t Q, const int4* __restrict__ pbox,
                                 int64_t N, int64_t* __restrict__ counts,
                                 const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cand)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= Q) return;
    const int4 a = qbox[q];
    int64_t cnt = 0, out = kWrite ? row_ptr[q] : 0;
    for (int64_t base = 0; base < N; base += 32) {
        const int64_t p = base + lane;
        bool hit = false;
        if (p < N) {
            const int4 b = pbox[p];
            hit = a.x < b.z && b.x < a.z && a.y < b.w && b.y < a.w;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (kWrite && hit) cand[out + cnt + __popc(m & pmh_lanemask_lt())] = (int32_t)p;
        cnt += __popc(m);
    }
    if (!kWrite && lane == 0) counts[q] = cnt;
}

}  // namespace

extern "C" int pmh_bbox_join(pmh_ctx ctx, pmh_polys queries, pmh_polys db, int64_t* d_row_ptr,
                             int32_t* d_cand, int64_t cand_capacity, int64_t* h_total, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!queries || !db || !d_row_ptr || !h_total || cand_capacity < 0)
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Q = queries->n;
    *h_total = 0;
    if (Q == 0) {
        PMH_CUDA_TRY(cudaMemsetAsync(d_row_ptr, 0, sizeof(int64_t), s));
        return PMH_OK;
    }
    int64_t* counts = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_QUERY, sizeof(int64_t) * (size_t)Q, (void**)&counts));
    const unsigned blocks = (unsigned)((Q + 7) / 8);
    bbox_join_kernel<false><<<blocks, 256, 0, s>>>(queries->bbox, Q, db->bbox, db->n, counts, nullptr,
                                                   nullptr);
    PMH_LAUNCHED("bbox_join_kernel<count>");
    PMH_TRY(pmh_exclusive_scan_i64(ctx, counts, d_row_ptr, Q, s));
    PMH_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, d_row_ptr + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t total = ctx->h_pinned[0];
    *h_total = total;
    if (total > cand_capacity)
        return pmh_set_error(PMH_ERR_CAPACITY, "%lld pairs > capacity %lld", (long long)total,
                             (long long)cand_capacity);
    if (total == 0) return PMH_OK;
    if (!d_cand) return pmh_set_error(PMH_ERR_ARG, "null candidate buffer");
    bbox_join_kernel<true><<<blocks, 256, 0, s>>>(queries->bbox, Q, db->bbox, db->n, nullptr, d_row_ptr,
                                                  d_cand);
    PMH_LAUNCHED("bbox_join_kernel<fill>");
    return PMH_OK;
}

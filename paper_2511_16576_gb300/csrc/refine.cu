// refine.cu -- step A8: exact Jaccard refinement (Sec. 5.2 refinement phase;
// J = area(A n B) / area(A u B), Sec. 1).
//
// area(A n B) by Green's theorem: the boundary of A n B is made of the pieces
// of A's edges inside B and of B's edges inside A, and area = closed integral
// of x dy over it.  Along one edge the pieces need not be sorted: with
// F(t) = dy * (x0 t + dx t^2 / 2) (x dy integrated from the edge start to
// parameter t), an edge that starts inside contributes nothing at t = 0, every
// crossing where it enters the other polygon contributes -F(t), every exit
// +F(t), and an edge that ends inside adds F(1).  Every term is independent,
// so one warp sums them for one pair in any order: each crossing of an A edge
// with a B edge is met once and adds both edges' terms with one reciprocal, and
// the "ends inside" state of an edge is the start state of the next edge.
//
// Degenerate contacts (a vertex on an edge, overlapping collinear edges,
// identical polygons) are resolved by simulation of simplicity: A is taken as
// shifted by (e1, e2), 0 < e2 << e1 infinitesimal.  Every predicate is then
// decided exactly with int64 cross products (coordinates <= 2^20), and the
// area of the shifted configuration tends to the exact one.  The terms are
// fp64 in coordinates relative to B's first vertex.  GB300's fp64 rate is low,
// so the fp64 work is kept to the crossings (a few per edge) and one Newton
// reciprocal each.
#include <algorithm>
#include <climits>

#include "pmh_internal.cuh"

namespace {


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

// 1/D in double precision for an integer D != 0 (|D| < 2^44): a single-precision
// reciprocal as the start, then two Newton steps y <- y + y(1 - D y), each of
// which squares the relative error (2^-23 -> 2^-46 -> below double rounding).
// Cheaper on this GPU's narrow fp64 pipe than a correctly rounded division;
// the result is within a few units in the last place, far inside the 1e-9
// relative tolerance of the refinement.
__device__ __forceinline__ double recip(long long D)
{
    const double d = (double)D;
    double y = (double)(1.0f / (float)d);
    double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    e = fma(-d, y, 1.0);
    return fma(y, e, y);
}

// area(A n B) for one pair, by one warp; returned in every lane.
//  * end terms: edge e_i of the shifted A ends inside B iff its end vertex
//    a_{i+1} + e is inside B (the start state of the next edge), so each lane
//    tests its vertices and adds F(1) of the edge that ends there -- no crossing
//    parity per edge is needed; likewise for B's edges and A + e;
//  * crossings: each (A edge, B edge) pair that crosses is visited by one lane,
//    which adds both boundary terms from one reciprocal: with D = de x df,
//    t = Nt / D on e and u = Nu / D on f (Nt, Nu, D exact integers),
//    F_e(t) = dy t (x0e + dx t / 2) and F_f(u) = ey u (x0f + ex u / 2).
// boundary terms of one crossing, queued as (A edge i, B edge j): with
// D = de x df, t = Nt / D on e and u = Nu / D on f (Nt, Nu, D exact integers),
// F_e(t) = dy t (x0e + dx t / 2) and F_f(u) = ey u (x0f + ex u / 2), signed by
// the direction of the crossing
__device__ __forceinline__ double crossing_terms(const int2* __restrict__ A, int na, int sA,
                                                 const int2* __restrict__ B, int nb, int sB,
                                                 int2 org, uint2 ij)
{
    const int i = (int)ij.x, j = (int)ij.y;
    const int2 a = A[i], b = A[i + 1 == na ? 0 : i + 1];
    const int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
    const int s2 = side_of_shifted_point(c, d, b), s4 = side_of_point_to_shifted(a, b, d);
    const long long dx = b.x - a.x, dy = b.y - a.y, ex = d.x - c.x, ey = d.y - c.y;
    const long long D = dx * ey - dy * ex;
    const long long Nt = (long long)(c.x - a.x) * ey - (long long)(c.y - a.y) * ex;
    const long long Nu = (long long)(c.x - a.x) * dy - (long long)(c.y - a.y) * dx;
    // A's edge: entering B flips the sign; B's edge: entering the shifted A
    const double sa = (((s2 > 0) == (sB > 0)) ? -1.0 : 1.0) * (sA > 0 ? 1.0 : -1.0);
    const double sb = (((s4 > 0) == (sA > 0)) ? -1.0 : 1.0) * (sB > 0 ? 1.0 : -1.0);
    const double r = recip(D);  // D != 0: the edges cross at one point
    const double t = (double)Nt * r, u = (double)Nu * r;
    const double fa = (double)dy * t * ((double)(a.x - org.x) + 0.5 * (double)dx * t);
    const double fb = (double)ey * u * ((double)(c.x - org.x) + 0.5 * (double)ex * u);
    return sa * fa + sb * fb;
}

// One warp's part of area(A n B) for a pair worked on by two warps (wip = 0, 1):
// the end terms of A's vertices (wip 0) or of B's (wip 1), and the crossings of
// the A edges in the 32-edge groups of its parity; summed over the warp.
__device__ double warp_intersection_area(const int2* __restrict__ A, int na, int sA,
                                         const int2* __restrict__ B, int nb, int sB,
                                         uint2* cq /* [64] */, int lane, int wip)
{
    const int2 org = B[0];
    double acc = 0;
    // end terms of A's edges: vertex a_i + e inside B closes edge i-1
    for (int i = wip == 0 ? lane : na; i < na; i += 32) {
        const int2 a = A[i];
        unsigned in = 0;
        for (int j = 0; j < nb; ++j) {
            const int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
            if ((c.y > a.y) != (d.y > a.y)) {
                const long long cr = cross3(c, d, a);
                in ^= (cr != 0) & ((cr > 0) == (d.y > c.y));
            }
        }
        if (in) {
            const int2 p = A[i == 0 ? na - 1 : i - 1];
            const double x0 = (double)(p.x - org.x), dx = (double)(a.x - p.x), dy = (double)(a.y - p.y);
            acc += (sA > 0 ? 1.0 : -1.0) * dy * (x0 + 0.5 * dx);
        }
    }
    // end terms of B's edges: vertex c_j - e inside A closes edge j-1
    for (int j = wip == 1 ? lane : nb; j < nb; j += 32) {
        const int2 c = B[j];
        unsigned in = 0;
        for (int i = 0; i < na; ++i) {
            const int2 a = A[i], b = A[i + 1 == na ? 0 : i + 1];
            if ((a.y >= c.y) != (b.y >= c.y)) {
                const long long cr = cross3(a, b, c);
                in ^= (cr == 0) | ((cr > 0) == (b.y > a.y));
            }
        }
        if (in) {
            const int2 p = B[j == 0 ? nb - 1 : j - 1];
            const double x0 = (double)(p.x - org.x), ex = (double)(c.x - p.x), ey = (double)(c.y - p.y);
            acc += (sB > 0 ? 1.0 : -1.0) * ey * (x0 + 0.5 * ex);
        }
    }
    // crossings: the lanes find them with integer predicates only and queue them
    // (edge indices); the fp64 terms are then evaluated 32 at a time, one
    // crossing per lane, so the narrow fp64 pipe never runs a mostly idle warp
    const unsigned full = 0xffffffffu;
    int nq = 0;  // warp-uniform queue length (< 32 between iterations)
    for (int i0 = 32 * wip; i0 < na; i0 += 64) {
        const int i = i0 + lane;
        int2 a = make_int2(0, 0), b = make_int2(0, 0);
        bool live = i < na;
        if (live) {
            a = A[i];
            b = A[i + 1 == na ? 0 : i + 1];
            live = a.x != b.x || a.y != b.y;
        }
        const int ax0 = min(a.x, b.x), ax1 = max(a.x, b.x), ay0 = min(a.y, b.y), ay1 = max(a.y, b.y);
        for (int j = 0; j < nb; ++j) {
            bool hit = false;
            if (live) {
                const int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
                if (!(max(ax0, min(c.x, d.x)) > min(ax1, max(c.x, d.x)) ||
                      max(ay0, min(c.y, d.y)) > min(ay1, max(c.y, d.y)) || (c.x == d.x && c.y == d.y))) {
                    hit = side_of_shifted_point(c, d, a) != side_of_shifted_point(c, d, b) &&
                          side_of_point_to_shifted(a, b, c) != side_of_point_to_shifted(a, b, d);
                }
            }
            const unsigned bal = __ballot_sync(full, hit);
            if (bal) {
                if (hit) cq[nq + __popc(bal & pmh_lanemask_lt())] = make_uint2((uint32_t)i, (uint32_t)j);
                nq += __popc(bal);
                __syncwarp();
                if (nq >= 32) {
                    acc += crossing_terms(A, na, sA, B, nb, sB, org, cq[lane]);
                    nq -= 32;
                    const uint2 rest = lane < nq ? cq[32 + lane] : make_uint2(0u, 0u);
                    __syncwarp();
                    if (lane < nq) cq[lane] = rest;
                    __syncwarp();
                }
            }
        }
    }
    if (lane < nq) acc += crossing_terms(A, na, sA, B, nb, sB, org, cq[lane]);
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// y-slab lists of a ring v[0..n) (staged in shared memory or read from global
// memory; edge e = v[e] -> v[e+1 mod n]): edge e is listed in every slab of
// [y0 + s*2^sh, y0 + (s+1)*2^sh) that its closed y-range meets, 128 slabs (four
// per lane).  Returns false (warp-uniform) if more than kRefSlabCap references
// would be needed.
constexpr int kRefSlabs = 128;
constexpr int kSlabsPerLane = kRefSlabs / 32;
constexpr int kRefSlabCap = 2048;
struct RefSlabs {
    uint16_t ids[kRefSlabCap];
    uint16_t beg[kRefSlabs + 2];
    int cnt[kRefSlabs];
    int y0, sh;
    int x0, x1;  // the ring's x-range
};

__device__ __forceinline__ bool build_ref_slabs(const int2* v, int n, RefSlabs& L, int lane)
{
    int y0 = INT_MAX, y1 = INT_MIN, x0 = INT_MAX, x1 = INT_MIN;
    for (int e = lane; e < n; e += 32) {
        const int2 u = v[e];
        y0 = min(y0, u.y);
        y1 = max(y1, u.y);
        x0 = min(x0, u.x);
        x1 = max(x1, u.x);
    }
    y0 = __reduce_min_sync(0xffffffffu, y0);
    y1 = __reduce_max_sync(0xffffffffu, y1);
    x0 = __reduce_min_sync(0xffffffffu, x0);
    x1 = __reduce_max_sync(0xffffffffu, x1);
    int sh = 0;
    while (((y1 - y0) >> sh) >= kRefSlabs) ++sh;
#pragma unroll
    for (int u = 0; u < kSlabsPerLane; ++u) L.cnt[kSlabsPerLane * lane + u] = 0;
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        const int2 a = v[e], b = v[e + 1 == n ? 0 : e + 1];
        const int s0 = (min(a.y, b.y) - y0) >> sh, s1 = (max(a.y, b.y) - y0) >> sh;
        for (int q = s0; q <= s1; ++q) atomicAdd(&L.cnt[q], 1);
    }
    __syncwarp();
    int c[kSlabsPerLane], mine = 0;
#pragma unroll
    for (int u = 0; u < kSlabsPerLane; ++u) {
        c[u] = L.cnt[kSlabsPerLane * lane + u];
        mine += c[u];
    }
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > kRefSlabCap) return false;
    const int excl = incl - mine;
    {
        int run = excl;
#pragma unroll
        for (int u = 0; u < kSlabsPerLane; ++u) {
            L.beg[kSlabsPerLane * lane + u] = (uint16_t)run;
            run += c[u];
        }
    }
    if (lane == 31) L.beg[kRefSlabs] = (uint16_t)total;
    if (lane == 0) {
        L.y0 = y0;
        L.sh = sh;
        L.x0 = x0;
        L.x1 = x1;
    }
    __syncwarp();
    {
        int run = excl;
#pragma unroll
        for (int u = 0; u < kSlabsPerLane; ++u) {
            L.cnt[kSlabsPerLane * lane + u] = run;
            run += c[u];
        }
    }
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        const int2 a = v[e], b = v[e + 1 == n ? 0 : e + 1];
        const int s0 = (min(a.y, b.y) - y0) >> sh, s1 = (max(a.y, b.y) - y0) >> sh;
        for (int q = s0; q <= s1; ++q) L.ids[atomicAdd(&L.cnt[q], 1)] = (uint16_t)e;
    }
    __syncwarp();
    return true;
}

// area(A n B) as warp_intersection_area, for staged rings with slab lists: a
// vertex test reads only the other ring's slab of the vertex's y, and an A edge
// meets only the B edges listed in the slabs its y-range spans (each pair once:
// in the first of those slabs that also lists the B edge).
__device__ double warp_intersection_area_slabs(const int2* __restrict__ A, int na, int sA,
                                               const RefSlabs& LA, const int2* __restrict__ B, int nb,
                                               int sB, const RefSlabs& LB, uint2* cq, int lane, int wip)
{
    const int2 org = B[0];
    const unsigned full = 0xffffffffu;
    double acc = 0;
    const int ya0 = LA.y0, ya1 = LA.y0 + (kRefSlabs << LA.sh) - 1;
    const int yb0 = LB.y0, yb1 = LB.y0 + (kRefSlabs << LB.sh) - 1;
    // end terms of A's edges: vertex a_i + e inside B closes edge i-1 (a vertex strictly
    // left or right of B's x-range sees an even number of B's crossings: outside)
    for (int i = wip == 0 ? lane : na; i < na; i += 32) {
        const int2 a = A[i];
        unsigned in = 0;
        if (a.y >= yb0 && a.y <= yb1 && a.x >= LB.x0 && a.x <= LB.x1) {
            const int q = (a.y - yb0) >> LB.sh;
            for (int k = LB.beg[q]; k < LB.beg[q + 1]; ++k) {
                const int j = LB.ids[k];
                const int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
                if ((c.y > a.y) != (d.y > a.y)) {
                    const long long cr = cross3(c, d, a);
                    in ^= (cr != 0) & ((cr > 0) == (d.y > c.y));
                }
            }
        }
        if (in) {
            const int2 p = A[i == 0 ? na - 1 : i - 1];
            const double x0 = (double)(p.x - org.x), dx = (double)(a.x - p.x), dy = (double)(a.y - p.y);
            acc += (sA > 0 ? 1.0 : -1.0) * dy * (x0 + 0.5 * dx);
        }
    }
    // end terms of B's edges: vertex c_j - e inside A closes edge j-1
    for (int j = wip == 1 ? lane : nb; j < nb; j += 32) {
        const int2 c = B[j];
        unsigned in = 0;
        if (c.y >= ya0 && c.y <= ya1 && c.x >= LA.x0 && c.x <= LA.x1) {
            const int q = (c.y - ya0) >> LA.sh;
            for (int k = LA.beg[q]; k < LA.beg[q + 1]; ++k) {
                const int i = LA.ids[k];
                const int2 a = A[i], b = A[i + 1 == na ? 0 : i + 1];
                if ((a.y >= c.y) != (b.y >= c.y)) {
                    const long long cr = cross3(a, b, c);
                    in ^= (cr == 0) | ((cr > 0) == (b.y > a.y));
                }
            }
        }
        if (in) {
            const int2 p = B[j == 0 ? nb - 1 : j - 1];
            const double x0 = (double)(p.x - org.x), ex = (double)(c.x - p.x), ey = (double)(c.y - p.y);
            acc += (sB > 0 ? 1.0 : -1.0) * ey * (x0 + 0.5 * ex);
        }
    }
    // crossings, queued and evaluated 32 at a time as in warp_intersection_area
    int nq = 0;
    for (int i0 = 32 * wip; i0 < na; i0 += 64) {
        const int i = i0 + lane;
        int2 a = make_int2(0, 0), b = make_int2(0, 0);
        int k0 = 0, cntk = 0, q0 = 0;
        if (i < na) {
            a = A[i];
            b = A[i + 1 == na ? 0 : i + 1];
            const int lo = min(a.y, b.y), hi = max(a.y, b.y);
            // (an edge outside B's x-range meets no B edge)
            if ((a.x != b.x || a.y != b.y) && hi >= yb0 && lo <= yb1 && max(a.x, b.x) >= LB.x0 &&
                min(a.x, b.x) <= LB.x1) {
                q0 = (max(lo, yb0) - yb0) >> LB.sh;
                const int q1 = (min(hi, yb1) - yb0) >> LB.sh;
                k0 = LB.beg[q0];
                cntk = LB.beg[q1 + 1] - k0;
            }
        }
        const int ax0 = min(a.x, b.x), ax1 = max(a.x, b.x), ay0 = min(a.y, b.y), ay1 = max(a.y, b.y);
        const int steps = __reduce_max_sync(full, cntk);
        int q = q0;  // slab of list position k0 + t
        for (int t = 0; t < steps; ++t) {
            bool hit = false;
            int j = 0;
            if (t < cntk) {
                const int k = k0 + t;
                while (k >= LB.beg[q + 1]) ++q;
                j = LB.ids[k];
                const int2 c = B[j], d = B[j + 1 == nb ? 0 : j + 1];
                // this pair is visited once: in the first listed slab of both
                const int first = max(q0, (min(c.y, d.y) - yb0) >> LB.sh);
                if (q == first &&
                    !(max(ax0, min(c.x, d.x)) > min(ax1, max(c.x, d.x)) ||
                      max(ay0, min(c.y, d.y)) > min(ay1, max(c.y, d.y)) || (c.x == d.x && c.y == d.y))) {
                    hit = side_of_shifted_point(c, d, a) != side_of_shifted_point(c, d, b) &&
                          side_of_point_to_shifted(a, b, c) != side_of_point_to_shifted(a, b, d);
                }
            }
            const unsigned bal = __ballot_sync(full, hit);
            if (bal) {
                if (hit) cq[nq + __popc(bal & pmh_lanemask_lt())] = make_uint2((uint32_t)i, (uint32_t)j);
                nq += __popc(bal);
                __syncwarp();
                if (nq >= 32) {
                    acc += crossing_terms(A, na, sA, B, nb, sB, org, cq[lane]);
                    nq -= 32;
                    const uint2 rest = lane < nq ? cq[32 + lane] : make_uint2(0u, 0u);
                    __syncwarp();
                    if (lane < nq) cq[lane] = rest;
                    __syncwarp();
                }
            }
        }
    }
    if (lane < nq) acc += crossing_terms(A, na, sA, B, nb, sB, org, cq[lane]);
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(full, acc, o);
    return acc;
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

constexpr int kRefineWarps = 4;  // two pairs per block, two warps per pair
constexpr int kWarpVerts = 960;   // vertices of a pair's staging slice

// one pair's shared slice: the staged rings, a crossing queue per warp, both rings'
// slab lists, and the two warps' partial sums
struct RefPair {
    int2 sv[kWarpVerts];
    uint2 cq[2][64];
    RefSlabs sl[2];
    double part[2];
    long long e;
    int ok[2];
};

// the named barrier of pair slot g (0 or 1) of the block (barrier 0 is __syncthreads;
// immediate ids, so that the block holds three barriers)
__device__ __forceinline__ void pair_sync(int g)
{
    if (g == 0) asm volatile("bar.sync 1, 64;\n" ::: "memory");
    else asm volatile("bar.sync 2, 64;\n" ::: "memory");
}

// n vertices to shared memory by asynchronous 8-byte copies, 64 threads striding
// (the caller waits)
__device__ __forceinline__ void stage_ring(int2* dst, const int2* __restrict__ src, int n, int t)
{
    for (int i = t; i < n; i += 64) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + i) : "memory");
    }
}

// J of one pair by two warps (wip = 0, 1; every branch is uniform over both): both
// rings staged in the pair's shared slice when they fit, else read from global
// memory; warp 0 builds A's y-slab list and warp 1 B's, both when they fit their
// capacity, else every edge pair; the area's terms split between the warps, summed
// in a fixed order
__device__ double pair_jaccard(PairView A, PairView B, RefPair& P, int wip, int lane, int g)
{
    if (A.sgn == 0 || B.sgn == 0) return 0.0;
    const int2* a = A.v;
    const int2* b = B.v;
    // both rings staged when they fit the slice, else the one that fits (B first: its
    // edges are the inner loop of two of the three passes), else neither
    const bool sa = A.n + B.n <= kWarpVerts || (B.n > kWarpVerts && A.n <= kWarpVerts);
    const bool sb = A.n + B.n <= kWarpVerts || B.n <= kWarpVerts;
    if (sa || sb) {
        const int boff = sa ? A.n : 0;
        if (sa) stage_ring(P.sv, A.v, A.n, 32 * wip + lane);
        if (sb) stage_ring(P.sv + boff, B.v, B.n, 32 * wip + lane);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        pair_sync(g);
        if (sa) a = P.sv;
        if (sb) b = P.sv + boff;
    }
    const bool ok = build_ref_slabs(wip == 0 ? a : b, wip == 0 ? A.n : B.n, P.sl[wip], lane);
    if (lane == 0) P.ok[wip] = ok;
    pair_sync(g);
    const double part =
        P.ok[0] && P.ok[1]
            ? warp_intersection_area_slabs(a, A.n, A.sgn, P.sl[0], b, B.n, B.sgn, P.sl[1], P.cq[wip], lane, wip)
            : warp_intersection_area(a, A.n, A.sgn, b, B.n, B.sgn, P.cq[wip], lane, wip);
    if (lane == 0) P.part[wip] = part;
    pair_sync(g);
    const double inter = P.part[0] + P.part[1];
    const double uni = A.area + B.area - inter;
    return uni > 0 ? fmin(fmax(inter / uni, 0.0), 1.0) : 0.0;
}

__global__ void __launch_bounds__(kRefineWarps * 32, 7)
refine_pairs_kernel(const int2* __restrict__ qxy, const int64_t* __restrict__ qoff,
                    const int64_t* __restrict__ qarea2, const int4* __restrict__ qbox,
                    const int2* __restrict__ pxy, const int64_t* __restrict__ poff,
                    const int64_t* __restrict__ parea2, const int4* __restrict__ pbox,
                    const int32_t* __restrict__ ids, const int32_t* __restrict__ nlist, int m,
                    const int32_t* __restrict__ qid_list, int64_t n_pairs, double* __restrict__ out,
                    unsigned long long* __restrict__ ticket, const int64_t* __restrict__ d_n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = wid >> 1, wip = wid & 1;
    RefPair& P = reinterpret_cast<RefPair*>(smem_raw)[g];
    if (d_n && !qid_list) n_pairs = min(n_pairs, *d_n * (int64_t)m);  // lists of the live queries
    // persistent warp pairs pull pairs from a ticket: pair costs differ by orders of
    // magnitude (a query against its own source vs a neighbour it barely touches)
    for (;;) {
        if (wip == 0 && lane == 0) P.e = (long long)atomicAdd(ticket, 1ull);
        pair_sync(g);
        const int64_t e = P.e;
        if (e >= n_pairs) break;  // the same for both warps
        int64_t q;
        int32_t p;
        double j = -1.0;
        bool live = true;
        if (qid_list) {  // explicit pairs
            q = qid_list[e];
            p = ids[e];
        } else {         // top-m lists: pair e = (q, slot)
            q = e / m;
            const int slot = (int)(e - q * m);
            live = slot < nlist[q];
            p = live ? ids[e] : 0;
        }
        if (live) {
            // bounding boxes (half-open lattice boxes) without a common interior point:
            // an empty intersection, J = 0 exactly, as the full computation gives
            const int4 qa = qbox[q], pb = pbox[p];
            const bool apart = !(qa.x < pb.z && pb.x < qa.z && qa.y < pb.w && pb.y < qa.w);
            j = apart ? 0.0
                      : pair_jaccard(view(qxy, qoff, qarea2, q), view(pxy, poff, parea2, p), P, wip, lane, g);
        }
        if (wip == 0 && lane == 0) out[e] = j;
        pair_sync(g);  // the slice is free for the next pair
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
                                 int32_t* __restrict__ top_ids, double* __restrict__ top_j,
                                 const int64_t* __restrict__ d_n)
{
    extern __shared__ JKey s[];
    const int64_t q = blockIdx.x;
    if (d_n && q >= *d_n) return;  // past the live batch
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

// persistent grid (SM count x resident blocks) over the pairs
static int launch_refine(pmh_ctx ctx, const int2* qxy, const int64_t* qoff, const int64_t* qarea2,
                         const int4* qbox, pmh_polys db, const int32_t* ids, const int32_t* nlist, int m,
                         const int32_t* qid_list, int64_t n_pairs, double* out,
                         unsigned long long* ticket, const int64_t* d_n, cudaStream_t s)
{
    const size_t smem = sizeof(RefPair) * (kRefineWarps / 2);
    PMH_CUDA_TRY(cudaFuncSetAttribute(refine_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int per_sm = 0;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_pairs_kernel,
                                                               kRefineWarps * 32, smem));
    const int blocks = (int)std::min<int64_t>((n_pairs + 1) / 2,
                                              (int64_t)ctx->sm_count * std::max(per_sm, 1));
    PMH_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    refine_pairs_kernel<<<blocks, kRefineWarps * 32, smem, s>>>(
        qxy, qoff, qarea2, qbox, db->xy, db->offsets, db->area2, db->bbox, ids, nlist, m, qid_list,
        n_pairs, out, ticket, d_n);
    PMH_LAUNCHED("refine_pairs_kernel");
    return PMH_OK;
}

// context ticket slot of the refinement grid
constexpr int kRefineTicket = 6;

int pmh_launch_refine_topk(pmh_ctx ctx, const int2* qxy, const int64_t* qoff, const int64_t* qarea2,
                           const int4* qbox, pmh_polys db, const int32_t* ids, const int32_t* nlist, int64_t Q,
                           const int64_t* d_n, int32_t m, int32_t k, double* jv,
                           unsigned long long* ticket, int32_t* top_ids, double* top_j,
                           cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    PMH_TRY(launch_refine(ctx, qxy, qoff, qarea2, qbox, db, ids, nlist, m, nullptr, Q * m, jv, ticket, d_n,
                          s));
    int cap = 1;
    while (cap < m) cap <<= 1;
    const size_t smem = sizeof(JKey) * cap;
    topk_by_j_kernel<<<(unsigned)Q, 256, smem, s>>>(ids, nlist, jv, m, cap, k, top_ids, top_j, d_n);
    PMH_LAUNCHED("topk_by_j_kernel");
    return PMH_OK;
}

extern "C" int pmh_refine_topk(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_ids,
                               const int32_t* d_n, int64_t Q, int32_t m, int32_t k,
                               int32_t* d_top_ids, double* d_top_j, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!queries || !db || Q < 0 || Q > queries->n || m < 1 || m > 1024 || k < 1 || k > m ||
        (Q > 0 && (!d_ids || !d_n || !d_top_ids || !d_top_j)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (1 <= k <= m <= 1024)");
    if (Q == 0) return PMH_OK;
    double* jv = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_REFINE, sizeof(double) * (size_t)(Q * m), (void**)&jv));
    return pmh_launch_refine_topk(ctx, queries->xy, queries->offsets, queries->area2, queries->bbox, db,
                                  d_ids, d_n, Q,
                                  nullptr, m, k, jv, ctx->d_tickets + kRefineTicket, d_top_ids, d_top_j,
                                  (cudaStream_t)stream);
}

extern "C" int pmh_pair_jaccard(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_qid,
                                const int32_t* d_pid, int64_t n_pairs, double* d_j, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!queries || !db || n_pairs < 0 || (n_pairs > 0 && (!d_qid || !d_pid || !d_j)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    if (n_pairs == 0) return PMH_OK;
    return launch_refine(ctx, queries->xy, queries->offsets, queries->area2, queries->bbox, db, d_pid,
                         nullptr, 1, d_qid, n_pairs, d_j, ctx->d_tickets + kRefineTicket, nullptr,
                         (cudaStream_t)stream);
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

// sign_common.cuh -- device pieces shared by the two signing kernels (A1):
// the exact half-open membership test in its warp-cooperative and lane-local
// forms, the edge sources it reads (staged in shared memory with y-slab lists,
// or in global memory), the work counters and the stream walk.
#pragma once

#include "pmh_internal.cuh"

namespace {

constexpr int kSmemVerts = kStagedMaxVerts;  // vertices staged per warp (larger polygons read global)
constexpr int kSlabs = 32;       // horizontal slabs of a staged polygon
constexpr int kSlabCap = 512;    // (edge, slab) references of a staged polygon


// Stage a polygon's n vertices into shared memory, closed (dst[n] = dst[0]), with
// asynchronous 8-byte global-to-shared copies (cp.async: the data bypasses the
// registers); the warp waits for its copies and synchronises before returning.
__device__ __forceinline__ void stage_vertices(int2* dst, const int2* __restrict__ src, int n, int lane)
{
    for (int i = lane; i <= n; i += 32) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + (i == n ? 0 : i))
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
}

// Parity contribution of edge a->b to the half-open crossing test of lattice
// point (px, py): the edge counts iff it straddles y = py ((ay > py) != (by > py))
// and the int64 cross product (b - a) x (p - a) is non-zero with the sign of
// (by - ay), i.e. (bx-ax)(py-ay) > (px-ax)(by-ay) for an upward edge, < for a
// downward one.
__device__ __forceinline__ unsigned edge_parity(int2 a, int2 b, int px, int py)
{
    const bool st = (a.y > py) != (b.y > py);
    const long long l = (long long)(b.x - a.x) * (py - a.y);
    const long long r = (long long)(px - a.x) * (b.y - a.y);
    return st & (b.y > a.y ? l > r : l < r);
}

// Exact half-open membership of lattice point (px, py), warp-cooperative.
// Edge a->b counts iff (ay > py) != (by > py) and the int64 cross product
// (b - a) x (p - a) is non-zero with the sign of (by - ay).
__device__ __forceinline__ bool warp_inside(const int2* __restrict__ v, int n, int px, int py,
                                            int lane)
{
    unsigned par = 0;
    for (int e = lane; e < n; e += 32) {
        int2 a = v[e];
        int2 b = v[e + 1 == n ? 0 : e + 1];
        bool st = (a.y > py) != (b.y > py);
        if (st) {
            long long cr = (long long)(b.x - a.x) * (py - a.y) - (long long)(px - a.x) * (b.y - a.y);
            par ^= (cr != 0) & ((cr > 0) == (b.y > a.y));
        }
    }
    return __popc(__ballot_sync(0xffffffffu, par)) & 1;
}

// Algorithmic work of one warp (warp-uniform counts): stream points the walk
// examined up to its result, grid cells and index entries read by the indexed
// form, bbox candidates it ordered, and edges tested by the exact membership.
struct Work {
    unsigned long long walk = 0, cells = 0, entries = 0, cand = 0, edges = 0, masked = 0;
    unsigned long long lane_edges = 0;  // per lane (lane-parallel tests), summed at the end
};

// The same counters compiled away, for launches that do not report their work: every
// function below takes its counters as a template parameter W (Work or NoWork).
struct Sink {
    __device__ __forceinline__ Sink& operator+=(unsigned long long) { return *this; }
    __device__ __forceinline__ Sink& operator++() { return *this; }
    __device__ __forceinline__ Sink operator++(int) { return *this; }
    __device__ __forceinline__ operator unsigned long long() const { return 0ull; }
};
struct NoWork {
    Sink walk, cells, entries, cand, edges, masked, lane_edges;
};

// Exact membership through the polygon's y-slab index: only the edges listed
// for the slab holding py can straddle the line y = py.
__device__ __forceinline__ bool warp_inside_slab(const int2* __restrict__ v, int n,
                                                 const int32_t* __restrict__ sp,
                                                 const int32_t* __restrict__ se, int slab_h,
                                                 int ymin, int px, int py, int lane, int& tested)
{
    const int s = (py - ymin) / slab_h;
    const int lo = sp[s], hi = sp[s + 1];
    tested = hi - lo;
    unsigned par = 0;
    for (int i = lo + lane; i < hi; i += 32) {
        int e = se[i];
        int2 a = v[e];
        int2 b = v[e + 1 == n ? 0 : e + 1];
        bool st = (a.y > py) != (b.y > py);
        if (st) {
            long long cr = (long long)(b.x - a.x) * (py - a.y) - (long long)(px - a.x) * (b.y - a.y);
            par ^= (cr != 0) & ((cr > 0) == (b.y > a.y));
        }
    }
    return __popc(__ballot_sync(0xffffffffu, par)) & 1;
}

struct AllEdges {
    const int2* v;
    int n;
    template <class W>
    __device__ __forceinline__ bool operator()(int px, int py, int lane, W& w) const
    {
        w.edges += n;
        return warp_inside(v, n, px, py, lane);
    }
};

struct SlabEdges {
    const int2* v;
    int n;
    const int32_t* sp;
    const int32_t* se;
    int slab_h, ymin;
    template <class W>
    __device__ __forceinline__ bool operator()(int px, int py, int lane, W& w) const
    {
        int tested = 0;
        const bool r = warp_inside_slab(v, n, sp, se, slab_h, ymin, px, py, lane, tested);
        w.edges += tested;
        return r;
    }
};

// Edges of a polygon staged in shared memory (v[0..n], v[n] = v[0]), binned by
// the horizontal slabs [y0 + s*2^sh, y0 + (s+1)*2^sh) that their y-range
// [min y, max y) meets: ids[beg[s] .. beg[s+1]) are the edges of slab s.  Only
// those edges can straddle a line y = py inside slab s.  Both the
// warp-cooperative test (lanes split the slab's edges) and the lane-local one
// (one point per lane) are exact.
struct StagedEdges {
    const int2* v;
    const uint8_t* ids;
    const uint16_t* beg;
    int y0, sh;
    template <class W>
    __device__ __forceinline__ bool operator()(int px, int py, int lane, W& w) const
    {
        const int s = (py - y0) >> sh;
        const int lo = beg[s], hi = beg[s + 1];
        w.edges += hi - lo;
        unsigned par = 0;
        for (int i = lo + lane; i < hi; i += 32) {
            const int e = ids[i];
            par ^= edge_parity(v[e], v[e + 1], px, py);
        }
        return __popc(__ballot_sync(0xffffffffu, par)) & 1;
    }
    template <class W>
    __device__ __forceinline__ bool lane_inside(int px, int py, W& w) const
    {
        const int s = (py - y0) >> sh;
        const int lo = beg[s], hi = beg[s + 1];
        w.lane_edges += hi - lo;
        unsigned par = 0;
        for (int i = lo; i < hi; ++i) {
            const int e = ids[i];
            par ^= edge_parity(v[e], v[e + 1], px, py);
        }
        return par;
    }
};

// Smallest slab shift with kSlabs slabs of height 2^sh covering h >= 1 rows.
__device__ __forceinline__ int staged_slab_shift(int h)
{
    int sh = 0;
    while (((h - 1) >> sh) >= kSlabs) ++sh;
    return sh;
}

// Bins the n edges of the staged polygon v (v[n] = v[0]) into the kSlabs slabs
// from y0 (counting pass, warp scan, filling pass; cnt is kSlabs ints of
// scratch).  Edges outside [y0, y0 + kSlabs*2^sh) are clipped away: no point
// of the clipped bounding box lies on their lines.  Horizontal edges straddle
// no line.  Returns false (warp-uniform) if more than kSlabCap references
// would be needed.
__device__ __forceinline__ bool build_staged_slabs(const int2* v, int n, int y0, int sh,
                                                   uint8_t* ids, uint16_t* beg, int* cnt, int lane)
{
    cnt[lane] = 0;
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        const int2 a = v[e], b = v[e + 1];
        const int s0 = max(0, (min(a.y, b.y) - y0) >> sh);
        const int s1 = min(kSlabs - 1, (max(a.y, b.y) - 1 - y0) >> sh);
        if (a.y != b.y)
            for (int s = s0; s <= s1; ++s) atomicAdd(&cnt[s], 1);
    }
    __syncwarp();
    const int c = cnt[lane];
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > kSlabCap) return false;
    beg[lane] = (uint16_t)(incl - c);
    if (lane == 31) beg[kSlabs] = (uint16_t)total;
    __syncwarp();
    cnt[lane] = incl - c;
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        const int2 a = v[e], b = v[e + 1];
        const int s0 = max(0, (min(a.y, b.y) - y0) >> sh);
        const int s1 = min(kSlabs - 1, (max(a.y, b.y) - 1 - y0) >> sh);
        if (a.y != b.y)
            for (int s = s0; s <= s1; ++s) ids[atomicAdd(&cnt[s], 1)] = (uint8_t)e;
    }
    __syncwarp();
    return true;
}

template <int U, class Inside, class W>
__device__ __forceinline__ uint32_t sign_walk(const Inside& inside, int x0, int y0, uint32_t w,
                                              uint32_t h, uint64_t sk, uint32_t T, int lane,
                                              W& work, uint32_t start);

// Membership through the polygon's coverage mask first: a candidate in a cell
// that no edge touches is decided by the cell's code; only boundary cells run
// the exact test.
template <class Inner>
struct Masked {
    Inner inner;
    const uint32_t* m;  // 16 words (row j), 2 bits per cell
    int x0, y0, cwl, chl;
    template <class W>
    __device__ __forceinline__ bool operator()(int px, int py, int lane, W& w) const
    {
        const uint32_t code = (m[(py - y0) >> chl] >> (2 * ((px - x0) >> cwl))) & 3u;
        if (code != 2u) {
            w.masked += 1;
            return code == 1u;
        }
        return inner(px, py, lane, w);
    }
};

// One hash of one polygon; every lane returns the same value.  U points per
// lane per round: one round covers 32 * U consecutive stream indices.
template <int U, class Inside, class W>
__device__ __forceinline__ uint32_t sign_one_t(const Inside& inside, int x0, int y0, uint32_t w,
                                               uint32_t h, uint64_t sk, uint32_t T, int lane,
                                               W& work, uint32_t start = 0)
{
    if (w == 0 || h == 0) return T;
    const uint32_t r = sign_walk<U>(inside, x0, y0, w, h, sk, T, lane, work, start);
    work.walk += (r < T ? r + 1 : T) - start;
    return r;
}

template <int U, class Inside, class W>
__device__ __forceinline__ uint32_t sign_walk(const Inside& inside, int x0, int y0, uint32_t w,
                                              uint32_t h, uint64_t sk, uint32_t T, int lane,
                                              W& work, uint32_t start)
{
    uint64_t z = sk + (uint64_t)(start + lane + 1) * PMH_GAMMA;
    const uint64_t step = 32ull * PMH_GAMMA;
    for (uint32_t i0 = start; i0 < T; i0 += 32u * U) {
        uint32_t pts[U];
        unsigned m = 0;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            uint32_t r = pmh_mix64_lo(z + (uint64_t)j * step);
            pts[j] = r;
            uint32_t dx = (r & 0xFFFFu) - (uint32_t)x0;
            uint32_t dy = (r >> 16) - (uint32_t)y0;
            m |= (unsigned)((dx < w) & (dy < h)) << j;
        }
        z += (uint64_t)U * step;
        if (!__any_sync(0xffffffffu, m)) continue;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            unsigned b = __ballot_sync(0xffffffffu, (m >> j) & 1u);
            while (b) {
                int l = __ffs(b) - 1;
                b &= b - 1;
                uint32_t i = i0 + (uint32_t)(j * 32 + l);
                if (i >= T) return T;
                uint32_t r = __shfl_sync(0xffffffffu, pts[j], l);
                if (inside((int)(r & 0xFFFFu), (int)(r >> 16), lane, work)) return i;
            }
        }
    }
    return T;
}

// The rare walks of the indexed form (a list that overflowed, or no inside
// candidate below the index limit) are kept out of line, so that the registers
// of the walk do not weigh on the gather and the lane-parallel tests.
template <int U, class Inside, class W>
__device__ __noinline__ uint32_t sign_resume(const Inside inside, int x0, int y0, uint32_t w,
                                             uint32_t h, uint64_t sk, uint32_t T, int lane,
                                             W* work, uint32_t start)
{
    W local;
    const uint32_t r = sign_one_t<U>(inside, x0, y0, w, h, sk, T, lane, local, start);
    work->walk += local.walk;
    work->cand += local.cand;
    work->edges += local.edges;
    work->masked += local.masked;
    return r;
}


__device__ __forceinline__ long long orient(int2 a, int2 b, long long px, long long py)
{
    return (long long)(b.x - a.x) * (py - a.y) - (long long)(b.y - a.y) * (px - a.x);
}

// does the closed segment a-b meet the closed rectangle [rx0, rx1] x [ry0, ry1]?
__device__ __forceinline__ bool seg_meets_rect(int2 a, int2 b, long long rx0, long long ry0,
                                               long long rx1, long long ry1)
{
    if (max(a.x, b.x) < rx0 || min(a.x, b.x) > rx1 || max(a.y, b.y) < ry0 || min(a.y, b.y) > ry1)
        return false;
    const long long o1 = orient(a, b, rx0, ry0), o2 = orient(a, b, rx1, ry0);
    const long long o3 = orient(a, b, rx0, ry1), o4 = orient(a, b, rx1, ry1);
    const bool all_pos = o1 > 0 && o2 > 0 && o3 > 0 && o4 > 0;
    const bool all_neg = o1 < 0 && o2 < 0 && o3 < 0 && o4 < 0;
    return !(all_pos || all_neg);
}

}  // namespace

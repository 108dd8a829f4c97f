// slabs.cu -- per-polygon y-slab edge index and cost order (part of step A0,
// used by the batching path of A1).
//
// The exact membership test of a point at height py only involves edges that
// straddle the horizontal line through it.  For a polygon with many vertices
// (coastline-like boundaries with up to 65,536 vertices) the y-range of its
// bounding box is cut into S equal slabs and every slab lists the edges whose
// row range [min(ay,by), max(ay,by)) meets it.  A test then reads one slab's
// list instead of all n edges; the parity of the crossings is order-independent,
// so the order inside a list does not matter.
//
// Layout (only polygons with n > kSlabMinVerts get slabs):
//   slab_info[p] = {slab_base, edge_base, S, slab_h | ymin}: see SlabInfo
//   slab_ptr[slab_base .. slab_base + S]  int32 offsets into the edge list
//   slab_edges[edge_base + ...]           int32 local edge ids (edge e = v_e -> v_e+1)
//
// The cost order sorts polygons by the expected number of stream points per
// hash, 2^32 / area (Theorem 2, E[h] = 1/S_p), largest first, so that the
// persistent signing grid starts the longest items first.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

__device__ __forceinline__ int slab_count_for(int n, int height)
{
    int s = n / 4;
    s = max(s, 1);
    s = min(s, max(height, 1));
    return min(s, 1 << 16);
}

// floor(x / h) by a multiply: with m = floor(2^40 / h) + 1 (slab_div_magic), x * m / 2^40
// exceeds x / h by less than x / 2^40 < 2^-18 for x < 2^22, which is below the gap 1/h
// between x / h and the next integer for every h < 2^18 (slab heights here are at most
// 2^21 / 64 for polygons above 256 vertices, or 1), so the floor is exact
__device__ __forceinline__ uint64_t slab_div_magic(int h) { return (1ull << 40) / (uint64_t)h + 1ull; }
__device__ __forceinline__ int slab_div(int x, uint64_t m) { return (int)(((uint64_t)x * m) >> 40); }

// y of the two end points of edges e0 + 32u + lane (u < 4) of the ring of n vertices at
// xy + b, four loads in flight per lane: an edge's end vertex is the next lane's start
// vertex (a shuffle); lane 31 and the closing edge read theirs
__device__ __forceinline__ void edge_ys(const int2* __restrict__ xy, int64_t b, int n, int e0, int lane,
                                        int (&ay)[4], int (&by)[4])
{
    int own[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = e0 + 32 * u + lane;
        const bool edge_end = e < n && (lane == 31 || e + 1 == n);
        ay[u] = e < n ? xy[b + e].y : 0;
        own[u] = edge_end ? xy[b + (e + 1 == n ? 0 : e + 1)].y : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = e0 + 32 * u + lane;
        const int nx = __shfl_down_sync(0xffffffffu, ay[u], 1);
        by[u] = (lane == 31 || e + 1 == n) ? own[u] : nx;
    }
}

// pass 1: sizes of every polygon's slab table and edge list
__global__ void slab_size_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
                                 int64_t n_polys, const int64_t* __restrict__ d_n, int min_verts,
                                 SlabInfo* __restrict__ info, int64_t* __restrict__ ptr_sizes,
                                 int64_t* __restrict__ edge_sizes)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // slots at or past the device-side count (d_n) get empty sizes
    const int64_t n_live = d_n ? min(n_polys, *d_n) : n_polys;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_polys;
         p += nwarps) {
        const int64_t b = p < n_live ? off[p] : 0;
        const int n = p < n_live ? (int)(off[p + 1] - b) : 0;
        if (n <= min_verts) {
            if (lane == 0) {
                info[p] = SlabInfo{0, 0, 0, 1, 0};
                ptr_sizes[p] = 0;
                edge_sizes[p] = 0;
            }
            continue;
        }
        int y0 = 0x7fffffff, y1 = -0x7fffffff - 1;
        // four loads in flight per lane
        for (int i0 = 0; i0 < n; i0 += 128) {
            int y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u + lane;
                y[u] = i < n ? xy[b + i].y : xy[b].y;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                y0 = min(y0, y[u]);
                y1 = max(y1, y[u]);
            }
        }
        y0 = __reduce_min_sync(0xffffffffu, y0);
        y1 = __reduce_max_sync(0xffffffffu, y1);
        const int height = y1 - y0;
        const int S = slab_count_for(n, height);
        const int h = max((height + S - 1) / S, 1);
        const uint64_t hm = slab_div_magic(h);
        long long entries = 0;
        for (int e0 = 0; e0 < n; e0 += 128) {
            int ay[4], by[4];
            edge_ys(xy, b, n, e0, lane, ay, by);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (e0 + 32 * u + lane >= n || ay[u] == by[u]) continue;
                const int lo = min(ay[u], by[u]) - y0, hi = max(ay[u], by[u]) - 1 - y0;
                entries += slab_div(hi, hm) - slab_div(lo, hm) + 1;
            }
        }
        for (int o = 16; o > 0; o >>= 1) entries += __shfl_xor_sync(0xffffffffu, entries, o);
        if (lane == 0) {
            info[p] = SlabInfo{0, 0, S, h, y0};
            ptr_sizes[p] = S + 1;
            edge_sizes[p] = entries;
        }
    }
}

// pass 2: per polygon (one warp) count, prefix-sum and fill the slab lists; the
// counters of a polygon of at most kFillSmemSlabs slabs live in the warp's shared
// slice, larger ones in the global cursor array
constexpr int kFillThreads = 256;
constexpr int kFillSmemSlabs = 512;
__global__ void __launch_bounds__(kFillThreads, 8) slab_fill_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
                                 int64_t n_polys, const int64_t* __restrict__ d_n, int min_verts,
                                 SlabInfo* __restrict__ info, const int64_t* __restrict__ ptr_base,
                                 const int64_t* __restrict__ edge_base, int32_t* __restrict__ slab_ptr,
                                 int64_t cap_ptr, int32_t* __restrict__ cursor,
                                 int32_t* __restrict__ slab_edges, int64_t cap_edges)
{
    __shared__ int scur[kFillThreads / 32][kFillSmemSlabs + 1];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (d_n) n_polys = min(n_polys, *d_n);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_polys;
         p += nwarps) {
        const int64_t b = off[p];
        const int n = (int)(off[p + 1] - b);
        if (n <= min_verts) continue;
        SlabInfo si = info[p];
        const int S = si.S, h = si.slab_h, y0 = si.ymin;
        const uint64_t hm = slab_div_magic(h);
        const int64_t pb = ptr_base[p], eb = edge_base[p];
        if (ptr_base[p + 1] > cap_ptr || edge_base[p + 1] > cap_edges) {
            // the lists do not fit the fixed buffers: this polygon is tested over all its edges
            if (lane == 0) info[p].S = 0;
            continue;
        }
        if (lane == 0) {
            info[p].slab_base = pb;
            info[p].edge_base = eb;
        }
        int32_t* sp = slab_ptr + pb;
        int32_t* cur = S <= kFillSmemSlabs ? scur[threadIdx.x >> 5] : cursor + pb;
        for (int s = lane; s <= S; s += 32) cur[s] = 0;
        __syncwarp();
        for (int e0 = 0; e0 < n; e0 += 128) {
            int ay[4], by[4];
            edge_ys(xy, b, n, e0, lane, ay, by);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (e0 + 32 * u + lane >= n || ay[u] == by[u]) continue;
                const int lo = slab_div(min(ay[u], by[u]) - y0, hm);
                const int hi = slab_div(max(ay[u], by[u]) - 1 - y0, hm);
                for (int s = lo; s <= hi; ++s) atomicAdd(&cur[s], 1);
            }
        }
        __syncwarp();
        __threadfence_block();
        // exclusive prefix over S + 1 entries, 32 at a time
        int carry = 0;
        for (int base = 0; base <= S; base += 32) {
            int s = base + lane;
            int v = s < S ? cur[s] : 0;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (s <= S) sp[s] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        __syncwarp();
        for (int s = lane; s <= S; s += 32) cur[s] = sp[s];
        __syncwarp();
        for (int e0 = 0; e0 < n; e0 += 128) {
            int ay[4], by[4];
            edge_ys(xy, b, n, e0, lane, ay, by);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + 32 * u + lane;
                if (e >= n || ay[u] == by[u]) continue;
                const int lo = slab_div(min(ay[u], by[u]) - y0, hm);
                const int hi = slab_div(max(ay[u], by[u]) - 1 - y0, hm);
                for (int s = lo; s <= hi; ++s) slab_edges[eb + atomicAdd(&cur[s], 1)] = e;
            }
        }
        __syncwarp();
    }
}

// cost key: expected stream points per hash ~ 2^33 / |area2|, as orderable float bits,
// complemented so that an ascending sort puts the most expensive polygon first
__global__ void cost_key_kernel(const int64_t* __restrict__ area2, int64_t n,
                                uint32_t* __restrict__ keys, int32_t* __restrict__ ids)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        long long a = area2[p];
        const float aa = (float)(a < 0 ? -a : a);
        const float cost = 8589934592.0f / fmaxf(aa, 1.0f);
        keys[p] = ~__float_as_uint(cost);  // positive floats order like their bits
        ids[p] = (int32_t)p;
    }
}

// Morton code of a point of the 2^16 lattice (x bits at even positions)
__device__ __forceinline__ uint32_t morton16(uint32_t x, uint32_t y)
{
    auto spread = [](uint32_t v) {
        v &= 0xFFFFu;
        v = (v | (v << 8)) & 0x00FF00FFu;
        v = (v | (v << 4)) & 0x0F0F0F0Fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    return spread(x) | (spread(y) << 1);
}

// class key: polygons of more than kChunkMinVerts vertices (class 2) first, by
// decreasing expected cost -- the signing launch splits them into 32-hash items
// and starts the longest first -- then the staged polygons of the walk form and
// the polygons above kStagedMaxVerts (class 1), by decreasing expected cost,
// then staged polygons of the indexed form (class 0) in Morton order of their
// box centres -- warps running at the same time then read nearby cells of the
// stream index, which keeps them in L2; counts classes 0 and 1 into n_cls[0],
// n_cls[1]
__global__ void class_key_kernel(const int4* __restrict__ bbox, const int64_t* __restrict__ area2,
                                 const int64_t* __restrict__ off, int64_t n,
                                 uint32_t* __restrict__ keys, int32_t* __restrict__ ids,
                                 unsigned long long* __restrict__ n_cls)
{
    unsigned long long c0 = 0, c1 = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const long long a = area2[p];
        const float aa = (float)(a < 0 ? -a : a);
        const float cost = 8589934592.0f / fmaxf(aa, 1.0f);
        const int4 bb = bbox[p];
        const int64_t nv = off[p + 1] - off[p];
        const int cls = nv > kChunkMinVerts ? 2
                        : (nv > kStagedMaxVerts || pmh_index_plan(bb, a).lim == 0) ? 1 : 0;
        uint32_t key;
        if (cls == 0) {
            const uint32_t cx = (uint32_t)min((bb.x + bb.z) >> 1, 65535);
            const uint32_t cy = (uint32_t)min((bb.y + bb.w) >> 1, 65535);
            key = (2u << 30) | (morton16(cx, cy) >> 2);
        } else {
            key = ((uint32_t)(2 - cls) << 30) | (~__float_as_uint(cost) >> 2);
        }
        keys[p] = key;
        ids[p] = (int32_t)p;
        c0 += cls == 0;
        c1 += cls == 1;
    }
    if (c0) atomicAdd(&n_cls[0], c0);
    if (c1) atomicAdd(&n_cls[1], c1);
}

}  // namespace

int pmh_build_slabs(pmh_polys P, cudaStream_t s)
{
    pmh_ctx ctx = P->ctx;
    if (P->n == 0) return PMH_OK;
    const int64_t n = P->n;
    if (cudaMalloc(&P->slab_info, sizeof(SlabInfo) * n) != cudaSuccess) {
        cudaGetLastError();
        return pmh_set_error(PMH_ERR_NOMEM, "slab info allocation failed");
    }
    if (P->max_n <= kSlabMinVerts) {
        PMH_CUDA_TRY(cudaMemsetAsync(P->slab_info, 0, sizeof(SlabInfo) * n, s));
        return PMH_OK;
    }
    int64_t* sizes = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_MISC, sizeof(int64_t) * (size_t)(2 * (n + 1)), (void**)&sizes));
    int64_t* ptr_sizes = sizes;
    int64_t* edge_sizes = sizes + (n + 1);
    int blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)ctx->sm_count * 16);
    slab_size_kernel<<<blocks, 256, 0, s>>>(P->xy, P->offsets, n, nullptr, kSlabMinVerts, P->slab_info,
                                            ptr_sizes, edge_sizes);
    PMH_LAUNCHED("slab_size_kernel");
    PMH_TRY(pmh_exclusive_scan_i64(ctx, ptr_sizes, ptr_sizes, n, s));
    PMH_TRY(pmh_exclusive_scan_i64(ctx, edge_sizes, edge_sizes, n, s));
    PMH_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, ptr_sizes + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned + 1, edge_sizes + n, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t n_ptr = ctx->h_pinned[0], n_edges = ctx->h_pinned[1];
    int32_t* cursor = nullptr;
    if (cudaMalloc(&P->slab_ptr, sizeof(int32_t) * std::max<int64_t>(n_ptr, 1)) != cudaSuccess ||
        cudaMalloc(&P->slab_edges, sizeof(int32_t) * std::max<int64_t>(n_edges, 1)) != cudaSuccess ||
        cudaMalloc(&cursor, sizeof(int32_t) * std::max<int64_t>(n_ptr, 1)) != cudaSuccess) {
        cudaGetLastError();
        if (cursor) cudaFree(cursor);
        return pmh_set_error(PMH_ERR_NOMEM, "slab index allocation failed (%lld entries)",
                             (long long)n_edges);
    }
    slab_fill_kernel<<<blocks, 256, 0, s>>>(P->xy, P->offsets, n, nullptr, kSlabMinVerts, P->slab_info,
                                            ptr_sizes, edge_sizes, P->slab_ptr, INT64_MAX, cursor,
                                            P->slab_edges, INT64_MAX);
    cudaError_t e = cudaGetLastError();
    g_pmh_launches.fetch_add(1);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(cursor);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return pmh_set_error(PMH_ERR_CUDA, "slab fill failed: %s",
                             cudaGetErrorString(e != cudaSuccess ? e : e2));
    return PMH_OK;
}

int pmh_build_cost_order(pmh_polys P, cudaStream_t s)
{
    pmh_ctx ctx = P->ctx;
    const int64_t n = P->n;
    if (n == 0) return PMH_OK;
    uint32_t* keys = nullptr;
    if (cudaMalloc(&P->order, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&keys, sizeof(uint32_t) * n) != cudaSuccess) {
        cudaGetLastError();
        if (keys) cudaFree(keys);
        return pmh_set_error(PMH_ERR_NOMEM, "cost order allocation failed");
    }
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->sm_count * 32);
    cost_key_kernel<<<blocks, 256, 0, s>>>(P->area2, n, keys, P->order);
    cudaError_t e = cudaGetLastError();
    g_pmh_launches.fetch_add(1);
    int rc = e == cudaSuccess ? pmh_radix_sort_u32(ctx, keys, P->order, n, 32, s)
                              : pmh_set_error(PMH_ERR_CUDA, "cost key: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc == PMH_OK && e2 != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "cost order: %s", cudaGetErrorString(e2));
    cudaFree(keys);
    if (rc != PMH_OK) {
        cudaFree(P->order);
        P->order = nullptr;
    }
    return rc;
}

int pmh_build_class_order(pmh_polys P, cudaStream_t s)
{
    pmh_ctx ctx = P->ctx;
    const int64_t n = P->n;
    if (n == 0) return PMH_OK;
    uint32_t* keys = nullptr;
    if (cudaMalloc(&keys, sizeof(uint32_t) * n) != cudaSuccess) {
        cudaGetLastError();
        return pmh_set_error(PMH_ERR_NOMEM, "class order allocation failed");
    }
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->sm_count * 32);
    cudaError_t e;
    int rc = PMH_OK;
    // the class order of the indexed form; the class counts follow the keys
    if (cudaMalloc(&P->order_cls, sizeof(int32_t) * n) != cudaSuccess) {
        cudaGetLastError();
        rc = pmh_set_error(PMH_ERR_NOMEM, "class order allocation failed");
    }
    unsigned long long* n_cls = nullptr;
    if (rc == PMH_OK && cudaMalloc(&n_cls, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        rc = pmh_set_error(PMH_ERR_NOMEM, "class count allocation failed");
    }
    if (rc == PMH_OK && cudaMemsetAsync(n_cls, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "memset failed");
    if (rc == PMH_OK) {
        class_key_kernel<<<blocks, 256, 0, s>>>(P->bbox, P->area2, P->offsets, n, keys, P->order_cls, n_cls);
        g_pmh_launches.fetch_add(1);
        e = cudaGetLastError();
        rc = e == cudaSuccess ? pmh_radix_sort_u32(ctx, keys, P->order_cls, n, 32, s)
                              : pmh_set_error(PMH_ERR_CUDA, "class key: %s", cudaGetErrorString(e));
    }
    if (rc == PMH_OK &&
        cudaMemcpyAsync(ctx->h_pinned, n_cls, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "class count copy failed");
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc == PMH_OK && e2 != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "class order: %s", cudaGetErrorString(e2));
    if (rc == PMH_OK) {
        P->n_indexed = ctx->h_pinned[0];
        P->n_whole_cost = ctx->h_pinned[1];
    }
    if (n_cls) cudaFree(n_cls);
    cudaFree(keys);
    return rc;
}

// y-slab lists of a batch on fixed, caller-owned buffers, with no host
// synchronisation (for a captured pipeline): sizes per slot (zero past *d_n),
// two exclusive scans, and the lists of every polygon whose lists fit the
// buffers (slab_ptr: cap_ptr entries; slab_edges: cap_edges entries); a polygon
// whose lists do not fit gets S = 0 and is tested over all its edges.
// sizes: 2 * (max_polys + 1) entries; sums: 2 * pmh_scan_sums_size(max_polys).
int pmh_launch_slabs_fixed(pmh_ctx ctx, const int2* xy, const int64_t* off, int64_t max_polys,
                           const int64_t* d_n, SlabInfo* info, int64_t* sizes, int64_t* sums,
                           int32_t* slab_ptr, int64_t cap_ptr, int32_t* cursor, int32_t* slab_edges,
                           int64_t cap_edges, cudaStream_t s)
{
    if (max_polys <= 0) return PMH_OK;
    int64_t* ptr_sizes = sizes;
    int64_t* edge_sizes = sizes + (max_polys + 1);
    const int blocks = (int)std::min<int64_t>((max_polys + 7) / 8, (int64_t)ctx->sm_count * 16);
    slab_size_kernel<<<blocks, 256, 0, s>>>(xy, off, max_polys, d_n, kSlabMinVerts, info, ptr_sizes,
                                            edge_sizes);
    PMH_LAUNCHED("slab_size_kernel");
    PMH_TRY(pmh_exclusive_scan_i64(ctx, ptr_sizes, ptr_sizes, max_polys, s, sums));
    PMH_TRY(pmh_exclusive_scan_i64(ctx, edge_sizes, edge_sizes, max_polys, s,
                                   sums + pmh_scan_sums_size(max_polys)));
    slab_fill_kernel<<<blocks, 256, 0, s>>>(xy, off, max_polys, d_n, kSlabMinVerts, info, ptr_sizes,
                                            edge_sizes, slab_ptr, cap_ptr, cursor, slab_edges,
                                            cap_edges);
    PMH_LAUNCHED("slab_fill_kernel");
    return PMH_OK;
}

// api.cu -- contexts, errors, scratch memory and polygon upload (step A0).
//
// A0 follows Sec. 3.1 of the paper (per-polygon local MBR) with the fixed
// 65536^2 lattice as the global MBR; it also computes twice the signed area
// (exact int64 shoelace) for the refinement and the reranker features.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>

#include "pmh_internal.cuh"

std::atomic<int64_t> g_pmh_launches{0};

static thread_local char g_err[512] = "";

int pmh_set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" const char* pmh_last_error(void) { return g_err; }
extern "C" int pmh_version(void) { return 10000; }
extern "C" int64_t pmh_launch_count(void) { return g_pmh_launches.load(); }

int pmh_check_device(pmh_ctx ctx)
{
    if (!ctx) return pmh_set_error(PMH_ERR_ARG, "null context");
    cudaGetLastError();  // a stale error of an earlier, unrelated call must not fail this one
    PMH_CUDA_TRY(cudaSetDevice(ctx->device));
    return PMH_OK;
}

int pmh_check_params(const pmh_params* p)
{
    if (!p) return pmh_set_error(PMH_ERR_ARG, "null params");
    if (p->K < 1 || p->K > 4096) return pmh_set_error(PMH_ERR_ARG, "K=%u not in [1,4096]", p->K);
    if (p->T < 1 || p->T > (1u << 31)) return pmh_set_error(PMH_ERR_ARG, "T=%u not in [1,2^31]", p->T);
    if (p->bands < 1 || p->bands > 128 || p->K % p->bands != 0 || p->rows != p->K / p->bands)
        return pmh_set_error(PMH_ERR_ARG, "bands=%u rows=%u do not split K=%u (bands <= 128)",
                             p->bands, p->rows, p->K);
    return PMH_OK;
}

int pmh_scratch(pmh_ctx ctx, int slot, size_t bytes, void** out)
{
    if (bytes == 0) bytes = 256;
    if (ctx->scratch_bytes[slot] < bytes) {
        if (ctx->scratch[slot]) {
            PMH_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(ctx->scratch[slot]);
            ctx->scratch[slot] = nullptr;
            ctx->scratch_bytes[slot] = 0;
        }
        size_t want = bytes + bytes / 4;
        if (cudaMalloc(&ctx->scratch[slot], want) != cudaSuccess) {
            cudaGetLastError();
            return pmh_set_error(PMH_ERR_NOMEM, "scratch allocation of %zu bytes failed", want);
        }
        ctx->scratch_bytes[slot] = want;
    }
    *out = ctx->scratch[slot];
    return PMH_OK;
}

extern "C" int pmh_create(pmh_ctx* out, int device)
{
    if (!out) return pmh_set_error(PMH_ERR_ARG, "null out");
    *out = nullptr;
    int count = 0;
    PMH_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return pmh_set_error(PMH_ERR_ARG, "device %d not in [0,%d)", device, count);
    cudaDeviceProp prop;
    PMH_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return pmh_set_error(PMH_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a",
                             device, prop.major, prop.minor);
    PMH_CUDA_TRY(cudaSetDevice(device));
    pmh_ctx c = new pmh_ctx_s();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    if (cudaMalloc(&c->d_status, 64 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_tickets, 64 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned, 64 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        pmh_destroy(c);
        return pmh_set_error(PMH_ERR_NOMEM, "context allocation failed");
    }
    cudaMemset(c->d_status, 0, 64 * sizeof(int));
    cudaMemset(c->d_tickets, 0, 64 * sizeof(unsigned long long));
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    *out = c;
    return PMH_OK;
}

extern "C" int pmh_destroy(pmh_ctx ctx)
{
    if (!ctx) return PMH_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < SCR_COUNT; ++i)
        if (ctx->scratch[i]) cudaFree(ctx->scratch[i]);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_tickets) cudaFree(ctx->d_tickets);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    for (cudaEvent_t e : ctx->sign_ev) cudaEventDestroy(e);
    for (int l = 0; l < kIndexLevels; ++l) {
        if (ctx->sindex.cell[l]) cudaFree(ctx->sindex.cell[l]);
        if (ctx->sindex.ent[l]) cudaFree(ctx->sindex.ent[l]);
    }
    delete ctx;
    return PMH_OK;
}

// ---------------------------------------------------------------------------
// A0: per-polygon preparation.  One warp per polygon: validation, bbox
// (clipped to the lattice domain, half-open), twice the signed area.
// status[0] |= 1 bad offsets, 2 < 3 vertices, 4 coordinate out of range;
// status[1] = max vertex count.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 6) prep_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
                            int64_t n_polys, const int64_t* __restrict__ d_n, int64_t n_vertices,
                            int4* __restrict__ bbox, int64_t* __restrict__ area2,
                            int* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    if (d_n) n_polys = min(n_polys, *d_n);
    int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int LIM = 1 << 20;
    int nmax = 0;  // largest vertex count of the warp's polygons (one atomic at the end)
    for (int64_t p = warp; p < n_polys; p += nwarps) {
        int64_t b = off[p], e = off[p + 1];
        int flags = 0;
        if (b < 0 || e > n_vertices || e < b) flags |= 1;
        int64_t n = e - b;
        if (n < 3) flags |= 2;
        if (flags) {
            if (lane == 0) {
                atomicOr(&status[0], flags);
                bbox[p] = make_int4(0, 0, 0, 0);
                area2[p] = 0;
            }
            continue;
        }
        int x0 = INT_MAX, y0 = INT_MAX, x1 = INT_MIN, y1 = INT_MIN;
        long long a2 = 0;
        // four vertices per lane in flight; edge i's end vertex is lane + 1's vertex
        // (a shuffle), lane 31 reads it
        for (int64_t i0 = 0; i0 < n; i0 += 128) {
            int2 v[4], w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + 32 * u + lane;
                v[u] = i < n ? xy[b + i] : xy[b];
                w[u] = lane == 31 && i < n ? xy[b + (i + 1 == n ? 0 : i + 1)] : v[u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + 32 * u + lane;
                const int wx = __shfl_down_sync(0xffffffffu, v[u].x, 1);
                const int wy = __shfl_down_sync(0xffffffffu, v[u].y, 1);
                if (lane < 31) w[u] = make_int2(wx, wy);
                if (i < n) {
                    if (i + 1 == n) w[u] = xy[b];
                    if (v[u].x < -LIM || v[u].x > LIM || v[u].y < -LIM || v[u].y > LIM) flags |= 4;
                    x0 = min(x0, v[u].x);
                    x1 = max(x1, v[u].x);
                    y0 = min(y0, v[u].y);
                    y1 = max(y1, v[u].y);
                    a2 += (long long)v[u].x * w[u].y - (long long)w[u].x * v[u].y;
                }
            }
        }
        x0 = __reduce_min_sync(0xffffffffu, x0);
        y0 = __reduce_min_sync(0xffffffffu, y0);
        x1 = __reduce_max_sync(0xffffffffu, x1);
        y1 = __reduce_max_sync(0xffffffffu, y1);
        flags = __reduce_or_sync(0xffffffffu, flags);
        for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        if (lane == 0) {
            if (flags) atomicOr(&status[0], flags);
            // clip to the lattice domain [0, 65536)
            int cx0 = max(x0, 0), cy0 = max(y0, 0), cx1 = min(x1, 65536), cy1 = min(y1, 65536);
            if (cx1 < cx0) cx1 = cx0;
            if (cy1 < cy0) cy1 = cy0;
            bbox[p] = make_int4(cx0, cy0, cx1, cy1);
            area2[p] = a2;
            nmax = max(nmax, (int)(n < INT_MAX ? n : INT_MAX));
        }
    }
    if (lane == 0 && nmax > 0) atomicMax(&status[1], nmax);
}

int pmh_launch_prep(int sm_count, const int2* xy, const int64_t* off, int64_t n_polys,
                    const int64_t* d_n, int64_t n_vertices, int4* bbox, int64_t* area2,
                    int* status, cudaStream_t s)
{
    if (n_polys <= 0) return PMH_OK;
    int blocks = (int)std::min<int64_t>((n_polys + 7) / 8, (int64_t)sm_count * 16);
    prep_kernel<<<blocks, 256, 0, s>>>(xy, off, n_polys, d_n, n_vertices, bbox, area2, status);
    PMH_LAUNCHED("prep_kernel");
    return PMH_OK;
}

// per-polygon reranker inputs: log2(area) / 32 and log2(vertex count) / 16 (polygons
// below the device-side count d_n, when given)
__global__ void poly_feat_kernel(const int64_t* __restrict__ area2, const int64_t* __restrict__ off,
                                 int64_t n, const int64_t* __restrict__ d_n, float2* __restrict__ out)
{
    if (d_n) n = min(n, *d_n);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const long long a2 = area2[p];
        const double a = 0.5 * (double)(a2 < 0 ? -a2 : a2);
        out[p] = make_float2(log2f((float)(a > 1.0 ? a : 1.0)) / 32.f,
                             log2f((float)(off[p + 1] - off[p])) / 16.f);
    }
}

// copy the arrays in, validate them and compute every per-polygon product (bbox,
// 2 x area, reranker inputs, slab lists, class order) into P's buffers
static int upload_fill(pmh_polys P, const int32_t* xy, const int64_t* offsets, bool host,
                       cudaStream_t s)
{
    pmh_ctx ctx = P->ctx;
    const int64_t n_polys = P->n, n_vertices = P->nv;
    cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (n_vertices > 0) e = cudaMemcpyAsync(P->xy, xy, sizeof(int2) * n_vertices, kind, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->offsets, offsets, sizeof(int64_t) * (n_polys + 1), kind, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return pmh_set_error(PMH_ERR_CUDA, "upload copy failed: %s", cudaGetErrorString(e));
    // offsets[0] and offsets[n] are checked by the kernel through b/e bounds
    if (n_polys > 0)
        PMH_TRY(pmh_launch_prep(ctx->sm_count, P->xy, P->offsets, n_polys, nullptr, n_vertices, P->bbox,
                                P->area2, ctx->d_status, s));
    int st[2] = {0, 0};
    e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pmh_set_error(PMH_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e));
    memcpy(st, ctx->h_pinned, sizeof(st));
    if (st[0] & 1) return pmh_set_error(PMH_ERR_RANGE, "offsets are not increasing / in range");
    if (st[0] & 2) return pmh_set_error(PMH_ERR_RANGE, "a polygon has fewer than 3 vertices");
    if (st[0] & 4) return pmh_set_error(PMH_ERR_RANGE, "a coordinate exceeds |2^20|");
    P->max_n = st[1];
    if (n_polys > 0) {
        int blocks = (int)std::min<int64_t>((n_polys + 255) / 256, (int64_t)ctx->sm_count * 32);
        poly_feat_kernel<<<blocks, 256, 0, s>>>(P->area2, P->offsets, n_polys, nullptr, P->feat);
        g_pmh_launches.fetch_add(1);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return pmh_set_error(PMH_ERR_CUDA, "feature kernel: %s", cudaGetErrorString(e));
    }
    PMH_TRY(pmh_build_slabs(P, s));
    return pmh_build_class_order(P, s);
}

int pmh_launch_poly_feat(int sm_count, const int64_t* area2, const int64_t* off, int64_t n,
                         const int64_t* d_n, float2* out, cudaStream_t s)
{
    if (n <= 0) return PMH_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count * 32);
    poly_feat_kernel<<<blocks, 256, 0, s>>>(area2, off, n, d_n, out);
    PMH_LAUNCHED("poly_feat_kernel");
    return PMH_OK;
}

static int upload_common(pmh_ctx ctx, const int32_t* xy, const int64_t* offsets, int64_t n_polys,
                         int64_t n_vertices, bool host, pmh_polys* out, void* stream)
{
    if (!out) return pmh_set_error(PMH_ERR_ARG, "null out");
    *out = nullptr;
    PMH_TRY(pmh_check_device(ctx));
    if (n_polys < 0 || n_polys >= (1ll << 31) || n_vertices < 0 || (!xy && n_vertices > 0) ||
        !offsets)
        return pmh_set_error(PMH_ERR_ARG, "bad polygon arguments (n_polys=%lld n_vertices=%lld)",
                             (long long)n_polys, (long long)n_vertices);
    pmh_polys P = new pmh_polys_s();
    P->ctx = ctx;
    P->device = ctx->device;
    P->n = n_polys;
    P->nv = n_vertices;
    const size_t np = (size_t)(n_polys > 0 ? n_polys : 1);
    if (cudaMalloc(&P->xy, sizeof(int2) * (size_t)(n_vertices > 0 ? n_vertices : 1)) != cudaSuccess ||
        cudaMalloc(&P->offsets, sizeof(int64_t) * (size_t)(n_polys + 1)) != cudaSuccess ||
        cudaMalloc(&P->bbox, sizeof(int4) * np) != cudaSuccess ||
        cudaMalloc(&P->area2, sizeof(int64_t) * np) != cudaSuccess ||
        cudaMalloc(&P->feat, sizeof(float2) * np) != cudaSuccess) {
        cudaGetLastError();
        pmh_polys_destroy(P);
        return pmh_set_error(PMH_ERR_NOMEM, "polygon allocation failed (%lld vertices)",
                             (long long)n_vertices);
    }
    const int rc = upload_fill(P, xy, offsets, host, (cudaStream_t)stream);
    if (rc != PMH_OK) {
        pmh_polys_destroy(P);
        return rc;
    }
    *out = P;
    return PMH_OK;
}

// the per-polygon products that a reload rebuilds (their sizes follow the data)
static void free_derived(pmh_polys p)
{
    void* bufs[] = {p->slab_info, p->slab_ptr, p->slab_edges, p->order, p->order_cls, p->mask};
    for (void* b : bufs)
        if (b) cudaFree(b);
    p->slab_info = nullptr;
    p->slab_ptr = p->slab_edges = nullptr;
    p->order = p->order_cls = nullptr;
    p->mask = nullptr;
    p->n_indexed = p->n_whole_cost = 0;
}

extern "C" int pmh_poly_reload(pmh_polys polys, const int32_t* xy, const int64_t* offsets,
                               int64_t n_polys, int64_t n_vertices, int host_memory, void* stream)
{
    if (!polys) return pmh_set_error(PMH_ERR_ARG, "null polygons");
    PMH_TRY(pmh_check_device(polys->ctx));
    if (n_polys != polys->n || n_vertices != polys->nv || (!xy && n_vertices > 0) || !offsets)
        return pmh_set_error(PMH_ERR_ARG, "reload needs the set's own sizes (%lld polygons, %lld "
                             "vertices; got %lld, %lld)", (long long)polys->n, (long long)polys->nv,
                             (long long)n_polys, (long long)n_vertices);
    cudaStream_t s = (cudaStream_t)stream;
    PMH_CUDA_TRY(cudaStreamSynchronize(s));  // no kernel of this stream may still read the old data
    free_derived(polys);
    return upload_fill(polys, xy, offsets, host_memory != 0, s);
}

extern "C" int pmh_poly_upload(pmh_ctx ctx, const int32_t* d_xy, const int64_t* d_offsets,
                               int64_t n_polys, int64_t n_vertices, pmh_polys* out, void* stream)
{
    return upload_common(ctx, d_xy, d_offsets, n_polys, n_vertices, false, out, stream);
}

extern "C" int pmh_poly_upload_host(pmh_ctx ctx, const int32_t* h_xy, const int64_t* h_offsets,
                                    int64_t n_polys, int64_t n_vertices, pmh_polys* out,
                                    void* stream)
{
    return upload_common(ctx, h_xy, h_offsets, n_polys, n_vertices, true, out, stream);
}

extern "C" int pmh_polys_info(pmh_polys p, int64_t* n_polys, int64_t* n_vertices)
{
    if (!p) return pmh_set_error(PMH_ERR_ARG, "null polygons");
    if (n_polys) *n_polys = p->n;
    if (n_vertices) *n_vertices = p->nv;
    return PMH_OK;
}

extern "C" int pmh_polys_prep(pmh_polys p, int32_t* d_bbox, int64_t* d_area2, void* stream)
{
    if (!p) return pmh_set_error(PMH_ERR_ARG, "null polygons");
    PMH_TRY(pmh_check_device(p->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    if (d_bbox && p->n)
        PMH_CUDA_TRY(cudaMemcpyAsync(d_bbox, p->bbox, sizeof(int4) * p->n, cudaMemcpyDeviceToDevice, s));
    if (d_area2 && p->n)
        PMH_CUDA_TRY(cudaMemcpyAsync(d_area2, p->area2, sizeof(int64_t) * p->n,
                                     cudaMemcpyDeviceToDevice, s));
    return PMH_OK;
}

extern "C" int pmh_polys_destroy(pmh_polys p)
{
    if (!p) return PMH_OK;
    cudaSetDevice(p->device);
    if (p->xy || p->offsets || p->bbox || p->area2) cudaDeviceSynchronize();
    void* bufs[] = {p->xy, p->offsets, p->bbox, p->area2, p->feat, p->slab_info, p->slab_ptr,
                    p->slab_edges, p->order, p->order_cls, p->mask};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete p;
    return PMH_OK;
}

// stream_index.cu -- the first M points of every hash's stream, bucketed by
// lattice cell (used by the indexed signing path of A1).
//
// Every polygon draws from the same K point streams (Sec. 3.2: fixed seeds per
// hash function), so the points themselves can be indexed once: for each hash
// k the points i < M are sorted (stably) by their cell in a G x G grid over the
// domain.  A polygon then reads only the cells under its bounding box, and in
// each cell only the points below an index limit L; the smallest such index
// whose point lies in the polygon is h_k exactly, because every point of the
// stream with index < L that lies in the bounding box is in one of those
// cells.  If no point below L hits, the ordinary walk continues from L.
//
// Layout: the entries are sorted by (hash k, cell c, stream index); entry e =
// (stream index, x | y << 16), one 8-byte load.  The list of (k, c) is
// [cell[c*K + k].x, cell[(c+1)*K + k].x) (cell-major records).  cell[.].y holds
// six 5-bit counts: the entries of the list below M, M/2, ..., M/32, so that a
// reader with limit L knows how many entries to read (those below the smallest
// level >= L) without reading past them.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

__global__ void stream_points_kernel(uint64_t seed, int K, int M, int shift, int gbits,
                                     uint32_t* __restrict__ keys, int32_t* __restrict__ vals)
{
    const int64_t total = (int64_t)K * M;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / M);
        const int i = (int)(t - (int64_t)k * M);
        const uint64_t sk = pmh_mix64(seed + (uint64_t)(k + 1) * PMH_GAMMA);
        const uint32_t r = pmh_mix64_lo(sk + (uint64_t)(i + 1) * PMH_GAMMA);
        const uint32_t x = r & 0xFFFFu, y = r >> 16;
        const uint32_t cell = ((y >> shift) << gbits) | (x >> shift);
        keys[t] = ((uint32_t)k << (2 * gbits)) | cell;
        vals[t] = i;
    }
}

__global__ void cell_count_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                  int64_t* __restrict__ counts)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(&counts[keys[e]]), 1ull);
}

__global__ void finish_index_kernel(const uint32_t* __restrict__ keys, const int32_t* __restrict__ vals,
                                    int64_t n, uint64_t seed, int gbits, uint2* __restrict__ ent)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(keys[e] >> (2 * gbits));
        const int i = vals[e];
        const uint64_t sk = pmh_mix64(seed + (uint64_t)(k + 1) * PMH_GAMMA);
        ent[e] = make_uint2((uint32_t)i, pmh_mix64_lo(sk + (uint64_t)(i + 1) * PMH_GAMMA));
    }
}

// cell records (cell-major) from the k-major list starts: start and the rank
// counts of each level; row G*G holds each hash's end.  *longest = longest list
__global__ void cell_record_kernel(const int64_t* __restrict__ starts, int K, int gbits,
                                   const uint2* __restrict__ ent, int M, uint2* __restrict__ cell,
                                   int* __restrict__ longest)
{
    const int64_t GG = (int64_t)1 << (2 * gbits);
    const int64_t n_cells = GG * K;
    int mine = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = c >> (2 * gbits), cl = c & (GG - 1);
        const uint32_t b = (uint32_t)starts[c], e = (uint32_t)starts[c + 1];
        mine = max(mine, (int)(e - b));
        uint32_t counts = 0;
        for (int t = 0; t < kRankLevels; ++t) {
            const uint32_t level = (uint32_t)M >> t;
            uint32_t cnt = 0;
            for (uint32_t i = b; i < e && ent[i].x < level; ++i) ++cnt;
            counts |= min(cnt, 31u) << (5 * t);
        }
        cell[cl * K + k] = make_uint2(b, counts);
        if (cl == GG - 1) cell[GG * K + k] = make_uint2(e, 0u);
    }
    if (mine) atomicMax(longest, mine);
}

}  // namespace

// One level: the first M points of every hash's stream on a 2^gbits-square grid.
// Allocates *cell and *ent; on failure frees what it allocated.
static int build_level(pmh_ctx ctx, const pmh_params* P, cudaStream_t s, int M, int gbits,
                       uint2** cell_out, uint2** ent_out, int* ranked)
{
    const int shift = 16 - gbits;
    const int64_t n = (int64_t)P->K * M;
    const int64_t n_cells = (int64_t)P->K << (2 * gbits);
    uint2 *cell = nullptr, *ent = nullptr;
    if (cudaMalloc(&cell, sizeof(uint2) * (n_cells + P->K)) != cudaSuccess ||
        cudaMalloc(&ent, sizeof(uint2) * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(cell);
        cudaFree(ent);
        return pmh_set_error(PMH_ERR_NOMEM, "stream index allocation failed");
    }
    uint32_t* keys = nullptr;
    int32_t* vals = nullptr;
    int64_t* counts = nullptr;
    if (cudaMalloc(&keys, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&vals, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&counts, sizeof(int64_t) * (n_cells + 2)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(keys);
        cudaFree(vals);
        cudaFree(cell);
        cudaFree(ent);
        return pmh_set_error(PMH_ERR_NOMEM, "stream index scratch allocation failed");
    }
    int* longest = reinterpret_cast<int*>(counts + n_cells + 1);
    int rc = PMH_OK;
    const int blocks = ctx->sm_count * 16;
    stream_points_kernel<<<blocks, 256, 0, s>>>(P->seed, (int)P->K, M, shift, gbits, keys, vals);
    g_pmh_launches.fetch_add(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = pmh_set_error(PMH_ERR_CUDA, "stream points: %s", cudaGetErrorString(e));
    int key_bits = 2 * gbits;
    while ((1ll << key_bits) < (int64_t)P->K << (2 * gbits)) ++key_bits;
    if (rc == PMH_OK) rc = pmh_radix_sort_u32(ctx, keys, vals, n, key_bits, s);
    if (rc == PMH_OK && cudaMemsetAsync(counts, 0, sizeof(int64_t) * (n_cells + 2), s) != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "memset failed");
    if (rc == PMH_OK) {
        cell_count_kernel<<<blocks, 256, 0, s>>>(keys, n, counts);
        g_pmh_launches.fetch_add(1);
        rc = pmh_exclusive_scan_i64(ctx, counts, counts, n_cells, s);
    }
    if (rc == PMH_OK) {
        finish_index_kernel<<<blocks, 256, 0, s>>>(keys, vals, n, P->seed, gbits, ent);
        g_pmh_launches.fetch_add(1);
        cell_record_kernel<<<blocks, 256, 0, s>>>(counts, (int)P->K, gbits, ent, M, cell, longest);
        g_pmh_launches.fetch_add(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = pmh_set_error(PMH_ERR_CUDA, "finish: %s", cudaGetErrorString(e));
    }
    if (rc == PMH_OK && cudaMemcpyAsync(ctx->h_pinned, longest, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                            cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "stream index: copy failed");
    cudaError_t e2 = cudaStreamSynchronize(s);
    const int longest_list = rc == PMH_OK ? (int)*reinterpret_cast<int*>(ctx->h_pinned) : 0;
    cudaFree(keys);
    cudaFree(vals);
    cudaFree(counts);
    if (rc == PMH_OK && e2 != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "stream index build: %s", cudaGetErrorString(e2));
    if (rc != PMH_OK) {
        cudaFree(cell);
        cudaFree(ent);
        return rc;
    }
    *cell_out = cell;
    *ent_out = ent;
    *ranked = longest_list <= 31;  // else the counts saturate: only the list ends are used
    return PMH_OK;
}

static StreamIndexView view_of(const StreamIndex& si)
{
    StreamIndexView v{};
    for (int l = 0; l < kIndexLevels; ++l)
        v.lv[l] = IndexLevelView{si.cell[l], si.ent[l], index_level_points(l), index_level_gbits(l),
                                 16 - index_level_gbits(l), si.ranked[l]};
    v.cell = si.cell[0];
    v.ent = si.ent[0];
    v.M = index_level_points(0);
    v.gbits = index_level_gbits(0);
    v.shift = 16 - index_level_gbits(0);
    v.ranked = si.ranked[0];
    v.K = si.K;
    return v;
}

static void free_index(StreamIndex& si)
{
    for (int l = 0; l < kIndexLevels; ++l) {
        cudaFree(si.cell[l]);
        cudaFree(si.ent[l]);
    }
    si = StreamIndex();
}

int pmh_stream_index_get(pmh_ctx ctx, const pmh_params* P, cudaStream_t s, StreamIndexView* out)
{
    StreamIndex& si = ctx->sindex;
    if (si.cell[0] && si.seed == P->seed && si.K == (int)P->K) {
        *out = view_of(si);
        return PMH_OK;
    }
    if (si.cell[0]) {
        cudaDeviceSynchronize();
        free_index(si);
    }
    StreamIndex fresh;
    int rc = PMH_OK;
    for (int l = 0; l < kIndexLevels && rc == PMH_OK; ++l)
        if (l == 0 || index_level_fits(l, (int)P->K))  // level 0 always fits (K <= 4096)
            rc = build_level(ctx, P, s, index_level_points(l), index_level_gbits(l), &fresh.cell[l],
                             &fresh.ent[l], &fresh.ranked[l]);
    if (rc != PMH_OK) {
        free_index(fresh);
        return rc;
    }
    fresh.seed = P->seed;
    fresh.K = (int)P->K;
    si = fresh;
    *out = view_of(si);
    return PMH_OK;
}

extern "C" int pmh_stream_index_build(pmh_ctx ctx, const pmh_params* params, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    StreamIndexView v;
    return pmh_stream_index_get(ctx, params, (cudaStream_t)stream, &v);
}

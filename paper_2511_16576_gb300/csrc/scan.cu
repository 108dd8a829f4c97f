// scan.cu -- device-wide exclusive scan and a stable LSD radix sort.
//
// Both are plain bandwidth-bound building blocks of the bucket index:
//  * scan: reduce-then-scan over 2048-element tiles (three launches);
//  * sort: 8-bit digits, per pass one histogram kernel (per-tile digit counts,
//    digit-major), one scan of the counts, one scatter kernel that ranks the
//    tile's items stably (warp match + per-warp digit counters in shared
//    memory) and writes them to their global slots.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    int64_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    if (total) *total = sh[nw - 1];
    __syncthreads();
    return before;
}

__global__ void scan_reduce_kernel(const int64_t* __restrict__ in, int64_t n,
                                   int64_t* __restrict__ sums)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    int64_t total;
    block_exclusive_scan(s, sh, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of sums[0..nb) in place by one block, sums[nb] = total
__global__ void scan_sums_kernel(int64_t* __restrict__ sums, int64_t nb)
{
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        int64_t v = idx < nb ? sums[idx] : 0;
        int64_t total;
        int64_t ex = block_exclusive_scan(v, sh, &total);
        if (idx < nb) sums[idx] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_apply_kernel(const int64_t* __restrict__ in, int64_t n,
                                  const int64_t* __restrict__ sums, int64_t* __restrict__ out)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t ex = block_exclusive_scan(s, sh, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = sums[gridDim.x];
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;  // per lane
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t n_tiles,
                  int64_t* __restrict__ counts /* [256][n_tiles] */)
{
    __shared__ int hist[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&hist[(keys[idx] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
        counts[(int64_t)d * n_tiles + blockIdx.x] = hist[d];
}

// One tile per block.  Each warp owns kSortItems * 32 consecutive items of the
// tile, processed in chunks of 32 consecutive items, and ranks them stably per
// digit; the tile is then reordered by digit in shared memory (stable), and
// written out in that order, so that consecutive threads store consecutive
// positions of one digit's run instead of 32 scattered words.
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                     uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n, int shift,
                     int64_t n_tiles, const int64_t* __restrict__ offsets /* [256][n_tiles] */)
{
    __shared__ int wcount[kSortWarps][256];
    __shared__ int64_t base_off[256];
    __shared__ int tile_start[256];
    __shared__ int wsum[kSortWarps];
    __shared__ uint32_t sk[kSortTile];
    __shared__ int32_t sv[kSortTile];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&wcount[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
        base_off[d] = offsets[(int64_t)d * n_tiles + blockIdx.x];
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    const int tile_n = (int)(n - tbase < kSortTile ? n - tbase : kSortTile);
    const int wbase = wid * (kSortItems * 32);
    uint32_t k[kSortItems];
    int32_t v[kSortItems];
    int rank[kSortItems];
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        const int t = wbase + c * 32 + lane;
        const bool ok = t < tile_n;
        k[c] = ok ? kin[tbase + t] : 0;
        v[c] = ok ? vin[tbase + t] : 0;
    }
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        const bool ok = wbase + c * 32 + lane < tile_n;
        const unsigned d = (k[c] >> shift) & 0xFF;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? d : 0x100u) & act;
        int r = 0;
        if (ok) {
            const int before = __popc(peers & pmh_lanemask_lt());
            const int leader = __ffs(peers) - 1;
            int old = 0;
            if (lane == leader) {
                old = wcount[wid][d];
                wcount[wid][d] = old + __popc(peers);
            }
            old = __shfl_sync(peers, old, leader);
            r = old + before;
        }
        rank[c] = r;
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the digit's total in the tile
    const int dd = threadIdx.x;  // kSortThreads == 256 digits
    int total = 0;
    for (int w = 0; w < kSortWarps; ++w) {
        const int t = wcount[w][dd];
        wcount[w][dd] = total;
        total += t;
    }
    // exclusive prefix of the totals over digits: the digit runs' starts in the tile
    int x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < wid; ++w) pre += wsum[w];
    tile_start[dd] = pre + x - total;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        if (wbase + c * 32 + lane < tile_n) {
            const unsigned d = (k[c] >> shift) & 0xFF;
            const int pos = tile_start[d] + wcount[wid][d] + rank[c];
            sk[pos] = k[c];
            sv[pos] = v[c];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < tile_n; j += kSortThreads) {
        const uint32_t key = sk[j];
        const unsigned d = (key >> shift) & 0xFF;
        const int64_t dst = base_off[d] + (j - tile_start[d]);
        kout[dst] = key;
        vout[dst] = sv[j];
    }
}

}  // namespace

int64_t pmh_scan_sums_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

int pmh_exclusive_scan_i64(pmh_ctx ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s,
                           int64_t* sums_buffer)
{
    if (n <= 0) {
        PMH_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return PMH_OK;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t* sums = sums_buffer;
    if (!sums)
        PMH_TRY(pmh_scratch(ctx, SCR_SCAN, sizeof(int64_t) * (size_t)(nb + 1), (void**)&sums));
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    PMH_LAUNCHED("scan_reduce_kernel");
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums, nb);
    PMH_LAUNCHED("scan_sums_kernel");
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums, out);
    PMH_LAUNCHED("scan_apply_kernel");
    return PMH_OK;
}

int pmh_radix_sort_u32(pmh_ctx ctx, uint32_t* keys, int32_t* vals, int64_t n, int key_bits,
                       cudaStream_t s)
{
    if (n <= 1) return PMH_OK;
    int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* k2 = nullptr;
    int32_t* v2 = nullptr;
    int64_t* counts = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_SORT_A, sizeof(uint32_t) * (size_t)n, (void**)&k2));
    PMH_TRY(pmh_scratch(ctx, SCR_SORT_B, sizeof(int32_t) * (size_t)n, (void**)&v2));
    PMH_TRY(pmh_scratch(ctx, SCR_SORT_HIST, sizeof(int64_t) * (size_t)(256 * n_tiles + 1),
                        (void**)&counts));
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = p * 8;
        radix_hist_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(ka, n, shift, n_tiles, counts);
        PMH_LAUNCHED("radix_hist_kernel");
        PMH_TRY(pmh_exclusive_scan_i64(ctx, counts, counts, 256 * n_tiles, s));
        radix_scatter_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift,
                                                                         n_tiles, counts);
        PMH_LAUNCHED("radix_scatter_kernel");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PMH_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        PMH_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return PMH_OK;
}

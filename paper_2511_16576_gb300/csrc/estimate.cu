// estimate.cu -- steps A5 (agreement estimate) and A6 (top-m selection).
//
// A5 follows Theorem 1: Pr[h_k(q) = h_k(p)] = J(q, p), so the fraction of
// agreeing positions estimates J.  The candidate pairs of all rows are cut into
// chunks of consecutive pairs that warps take in turn (rows range from a few
// candidates to thousands, so a block per row would leave the grid waiting on
// the longest); a warp reads both rows' K hashes as 16-byte vectors (512 bytes
// per row at K = 128, the query's from L1/L2); equality bits are gathered with
// shuffles, the count is a warp reduction, and the band-match bits and the
// reranker's features (A7) come from the same bits.
//
// A6 sorts each candidate row by a 64-bit key in shared memory (bitonic),
// keeping the first m: key = (K - count) << 32 | id for the plain form,
// or (~orderable(score)) << 32 | id for a learned score.
#include <cuda_bf16.h>

#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kMaxK = 4096;
constexpr int kAgreeWarps = 4;
constexpr int kAgreeChunk = 16;  // consecutive pairs per warp turn

// Warps take chunks of kAgreeChunk consecutive pairs (the row of the first by
// binary search over row_ptr, then stepping on).  Per pair: equality bits of the
// K hashes (16-byte loads when K % 4 == 0), the count (warp sum), the full-match
// bits of the first 32 bands and, optionally, the reranker's feature row.
__global__ void __launch_bounds__(kAgreeWarps * 32)
agree_rows_kernel(const uint32_t* __restrict__ qh, const uint32_t* __restrict__ ph,
                  const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cand, int64_t Q,
                  int64_t cap, int K, int bands, int rows, uint32_t T, uint16_t* __restrict__ count,
                  uint32_t* __restrict__ bandmask, __nv_bfloat16* __restrict__ feat, FeatSrc qf,
                  FeatSrc pf, const int* __restrict__ d_flags)
{
    __shared__ uint32_t eqbits[kAgreeWarps][kMaxK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (d_flags && *d_flags) return;  // failed validation or candidate overflow
    const int64_t total = min(row_ptr[Q], cap);
    const int64_t nwarps = (int64_t)gridDim.x * kAgreeWarps;
    for (int64_t ch = (int64_t)blockIdx.x * kAgreeWarps + wid; ch * kAgreeChunk < total; ch += nwarps) {
        const int64_t x0 = ch * kAgreeChunk, x1 = min(x0 + kAgreeChunk, total);
        // the row holding pair x0: the last q with row_ptr[q] <= x0
        int64_t lo = 0, hi = Q;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= x0) lo = mid;
            else hi = mid;
        }
        int64_t q = lo;
        for (int64_t x = x0; x < x1; ++x) {
            while (row_ptr[q + 1] <= x) ++q;
            const uint32_t* qs = qh + q * K;
            const int64_t p = cand[x];
            const uint32_t* bp = ph + p * K;
            int c = 0, lt = 0, gt = 0;  // lt / gt: hashes with h(q) < h(p) / h(q) > h(p)
            if ((K & 3) == 0) {
                const uint4* a4 = reinterpret_cast<const uint4*>(qs);
                const uint4* b4 = reinterpret_cast<const uint4*>(bp);
                for (int base = 0; base < K / 4; base += 32) {
                    const int i = base + lane;
                    unsigned bits = 0;
                    if (i < K / 4) {
                        const uint4 u = __ldg(a4 + i), v = __ldg(b4 + i);
                        bits = (unsigned)((u.x == v.x) & (u.x != T)) |
                               ((unsigned)((u.y == v.y) & (u.y != T)) << 1) |
                               ((unsigned)((u.z == v.z) & (u.z != T)) << 2) |
                               ((unsigned)((u.w == v.w) & (u.w != T)) << 3);
                        if (feat) {
                            lt += (u.x < v.x) + (u.y < v.y) + (u.z < v.z) + (u.w < v.w);
                            gt += (u.x > v.x) + (u.y > v.y) + (u.z > v.z) + (u.w > v.w);
                        }
                    }
                    c += __popc(bits);
                    // hash 4i+t is bit (4i+t) % 32 of word i / 8: OR eight lanes' nibbles
                    unsigned w0 = bits << ((lane & 7) * 4);
                    w0 |= __shfl_xor_sync(0xffffffffu, w0, 1);
                    w0 |= __shfl_xor_sync(0xffffffffu, w0, 2);
                    w0 |= __shfl_xor_sync(0xffffffffu, w0, 4);
                    if ((lane & 7) == 0 && i < K / 4) eqbits[wid][i >> 3] = w0;
                }
            } else {
                for (int base = 0; base < K; base += 32) {
                    const int i = base + lane;
                    const bool eq = i < K && qs[i] == bp[i] && qs[i] != T;
                    const unsigned bal = __ballot_sync(0xffffffffu, eq);
                    c += eq;
                    if (feat && i < K) {
                        lt += qs[i] < bp[i];
                        gt += qs[i] > bp[i];
                    }
                    if (lane == 0) eqbits[wid][base / 32] = bal;
                }
            }
            __syncwarp();
            c = __reduce_add_sync(0xffffffffu, c);
            if (feat) {
                lt = __reduce_add_sync(0xffffffffu, lt);
                gt = __reduce_add_sync(0xffffffffu, gt);
            }
            if (count && lane == 0) count[x] = (uint16_t)c;
            if (bandmask) {
                bool all = lane < bands;
                for (int t = 0; t < rows && all; ++t) {
                    const int k = lane * rows + t;
                    all = (eqbits[wid][k >> 5] >> (k & 31)) & 1u;
                }
                const unsigned m = __ballot_sync(0xffffffffu, all);
                if (lane == 0) bandmask[x] = m;
            }
            if (feat) {
                // group j = hashes j*g .. j*g+g-1 (g = K / 32) all equal
                const int g = K / 32;
                bool all = true;
                for (int t = 0; t < g && all; ++t) {
                    const int k = lane * g + t;
                    all = (eqbits[wid][k >> 5] >> (k & 31)) & 1u;
                }
                __nv_bfloat16* f = feat + x * 48;
                f[lane] = __float2bfloat16_rn(all ? 1.f : 0.f);
                if (lane < 16) {
                    float v = 0.f;
                    if (lane == 0) v = (float)c / (float)K;
                    if (lane == 1) v = qf.feat[q].x;
                    if (lane == 2) v = pf.feat[p].x;
                    if (lane == 3) v = qf.feat[q].y;
                    if (lane == 4) v = pf.feat[p].y;
                    if (lane == 5) v = (float)lt / (float)K;
                    if (lane == 6) v = (float)gt / (float)K;
                    if (lane == 7) {
                        // upper bound of J: the intersection is at most min(|q|, |p|, overlap of
                        // the two bounding boxes)
                        const int4 qb = qf.bbox[q], pb = pf.bbox[p];
                        const float ow = (float)max(0, min(qb.z, pb.z) - max(qb.x, pb.x));
                        const float oh = (float)max(0, min(qb.w, pb.w) - max(qb.y, pb.y));
                        const long long qa = qf.area2[q], pa = pf.area2[p];
                        const float a = 0.5f * (float)(qa < 0 ? -qa : qa);
                        const float bq = 0.5f * (float)(pa < 0 ? -pa : pa);
                        const float mn = fminf(fminf(a, bq), ow * oh);
                        const float den = a + bq - mn;
                        v = den > 0.f ? mn / den : 0.f;
                    }
                    f[32 + lane] = __float2bfloat16_rn(v);
                }
            }
            __syncwarp();
        }
    }
}

// orderable float bits: larger float -> larger unsigned
__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

constexpr int kTopThreads = 256;
constexpr int kTopChunk = 2048;  // new items merged per round

__device__ void bitonic_sort_u64(uint64_t* s, int n /* power of two */)
{
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    uint64_t a = s[i], b = s[l];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// one block per query; running top-m kept in s[0..m), new chunk appended
__global__ void __launch_bounds__(kTopThreads)
topm_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cand,
            const uint16_t* __restrict__ count, const float* __restrict__ score, int K, int m,
            int cap /* power of two >= m + kTopChunk */, int32_t* __restrict__ out_ids,
            int32_t* __restrict__ out_n, const int* __restrict__ d_flags)
{
    extern __shared__ uint64_t s[];
    const int64_t q = blockIdx.x;
    const bool failed = d_flags && *d_flags;
    const int64_t b = failed ? 0 : row_ptr[q], e = failed ? 0 : row_ptr[q + 1];
    int kept = 0;
    for (int64_t base = b; base < e; base += kTopChunk) {
        int take = (int)(e - base < kTopChunk ? e - base : kTopChunk);
        // sort only the occupied prefix, rounded up to a power of two (most lists are short)
        int sz = 2;
        while (sz < kept + take) sz <<= 1;
        for (int i = threadIdx.x; i < sz; i += blockDim.x) {
            uint64_t key = ~0ull;
            if (i >= kept && i < kept + take) {
                int64_t idx = base + (i - kept);
                uint32_t hi = score ? ~f2ord(score[idx]) : (uint32_t)(K - (int)count[idx]);
                key = ((uint64_t)hi << 32) | (uint32_t)cand[idx];
            } else if (i < kept) {
                key = s[i];
            }
            s[i] = key;
        }
        __syncthreads();
        bitonic_sort_u64(s, sz);
        kept = min(m, kept + take);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        out_ids[q * m + i] = i < kept ? (int32_t)(uint32_t)(s[i] & 0xFFFFFFFFu) : -1;
    if (threadIdx.x == 0) out_n[q] = kept;
}

// fixed-width lists (ids [Q][m], -1 padded, counts n[Q]) to compact CSR; rows at or
// past the device-side count d_n (optional) are empty
__global__ void list_counts_kernel(const int32_t* __restrict__ n, int64_t Q,
                                   const int64_t* __restrict__ d_n, int64_t* __restrict__ c)
{
    const int64_t live = d_n ? min(Q, *d_n) : Q;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x)
        c[q] = q < live ? n[q] : 0;
}

__global__ void list_copy_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ n,
                                 int64_t Q, int m, const int64_t* __restrict__ d_n,
                                 const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cand)
{
    if (d_n) Q = min(Q, *d_n);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < Q * m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / m;
        const int i = (int)(t - q * m);
        if (i < n[q]) cand[row_ptr[q] + i] = ids[t];
    }
}

}  // namespace

extern "C" int pmh_lists_to_csr(pmh_ctx ctx, const int32_t* d_ids, const int32_t* d_n, int64_t Q,
                                int32_t m, int64_t* d_row_ptr, int32_t* d_cand, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (Q < 0 || m < 1 || !d_row_ptr || (Q > 0 && (!d_ids || !d_n || !d_cand)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (Q == 0) {
        PMH_CUDA_TRY(cudaMemsetAsync(d_row_ptr, 0, sizeof(int64_t), s));
        return PMH_OK;
    }
    int64_t* counts = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_QUERY, sizeof(int64_t) * (size_t)Q, (void**)&counts));
    return pmh_launch_lists_to_csr(ctx, d_ids, d_n, Q, m, nullptr, counts, nullptr, d_row_ptr, d_cand, s);
}

int pmh_launch_lists_to_csr(pmh_ctx ctx, const int32_t* ids, const int32_t* n, int64_t Q, int32_t m,
                            const int64_t* d_q, int64_t* counts, int64_t* sums, int64_t* row_ptr,
                            int32_t* cand, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    const int blocks = (int)std::min<int64_t>((Q * m + 255) / 256, (int64_t)ctx->sm_count * 32);
    list_counts_kernel<<<blocks, 256, 0, s>>>(n, Q, d_q, counts);
    PMH_LAUNCHED("list_counts_kernel");
    PMH_TRY(pmh_exclusive_scan_i64(ctx, counts, row_ptr, Q, s, sums));
    list_copy_kernel<<<blocks, 256, 0, s>>>(ids, n, Q, m, d_q, row_ptr, cand);
    PMH_LAUNCHED("list_copy_kernel");
    return PMH_OK;
}

int pmh_launch_agree(pmh_ctx ctx, const uint32_t* qh, const uint32_t* ph, const int64_t* row_ptr,
                     const int32_t* cand, int64_t Q, int64_t cap, const pmh_params* P,
                     uint16_t* count, uint32_t* bandmask, const int* d_flags, cudaStream_t s)
{
    return pmh_launch_agree_features(ctx, qh, ph, row_ptr, cand, Q, cap, P, count, bandmask, nullptr,
                                     FeatSrc{}, FeatSrc{}, d_flags, s);
}

int pmh_launch_agree_features(pmh_ctx ctx, const uint32_t* qh, const uint32_t* ph,
                              const int64_t* row_ptr, const int32_t* cand, int64_t Q, int64_t cap,
                              const pmh_params* P, uint16_t* count, uint32_t* bandmask,
                              uint16_t* feat, FeatSrc qf, FeatSrc pf, const int* d_flags,
                              cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    const int blocks = ctx->sm_count * 16;  // persistent: pair chunks are handed out in turn
    agree_rows_kernel<<<blocks, kAgreeWarps * 32, 0, s>>>(
        qh, ph, row_ptr, cand, Q, cap, (int)P->K, (int)P->bands, (int)P->rows, P->T, count, bandmask,
        reinterpret_cast<__nv_bfloat16*>(feat), qf, pf, d_flags);
    PMH_LAUNCHED("agree_rows_kernel");
    return PMH_OK;
}

int pmh_launch_topm(const int64_t* row_ptr, const int32_t* cand, const uint16_t* count,
                    const float* score, int64_t Q, int32_t m, int32_t* out_ids, int32_t* out_n,
                    const int* d_flags, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    int cap = 1;
    while (cap < m + kTopChunk) cap <<= 1;
    size_t smem = sizeof(uint64_t) * cap;
    PMH_CUDA_TRY(cudaFuncSetAttribute(topm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    topm_kernel<<<(unsigned)Q, kTopThreads, smem, s>>>(row_ptr, cand, count, score, 4096, m, cap,
                                                       out_ids, out_n, d_flags);
    PMH_LAUNCHED("topm_kernel");
    return PMH_OK;
}

extern "C" int pmh_jaccard_estimate(pmh_ctx ctx, const uint32_t* d_qhashes,
                                    const uint32_t* d_dbhashes, const int64_t* d_row_ptr,
                                    const int32_t* d_cand, int64_t Q, const pmh_params* params,
                                    uint16_t* d_count, uint32_t* d_bandmask, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (Q < 0 || (Q > 0 && (!d_qhashes || !d_dbhashes || !d_row_ptr || !d_count)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    return pmh_launch_agree(ctx, d_qhashes, d_dbhashes, d_row_ptr, d_cand, Q, INT64_MAX, params,
                            d_count, d_bandmask, nullptr, (cudaStream_t)stream);
}

extern "C" int pmh_topm(pmh_ctx ctx, const int64_t* d_row_ptr, const int32_t* d_cand,
                        const uint16_t* d_count, const float* d_score, int64_t Q, int32_t m,
                        int32_t* d_out_ids, int32_t* d_out_n, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (Q < 0 || m < 1 || m > 1024 || (Q > 0 && (!d_row_ptr || !d_out_ids || !d_out_n)) ||
        (!d_count && !d_score))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (m in [1,1024])");
    if (Q > 0x7FFFFFFF) return pmh_set_error(PMH_ERR_ARG, "too many queries");
    return pmh_launch_topm(d_row_ptr, d_cand, d_count, d_score, Q, m, d_out_ids, d_out_n, nullptr,
                           (cudaStream_t)stream);
}

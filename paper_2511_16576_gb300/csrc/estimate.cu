// estimate.cu -- steps A5 (agreement estimate) and A6 (top-m selection).
//
// A5 follows Theorem 1: Pr[h_k(q) = h_k(p)] = J(q, p), so the fraction of
// agreeing positions estimates J.  One warp handles one (query, candidate)
// pair: the K hashes of both rows are read as 16-byte vectors (coalesced, 512
// bytes per row at K = 128), equality bits are gathered with ballots, the
// count is a warp reduction and the per-band full-match bits come from the
// same ballots.
//
// A6 sorts each candidate row by a 64-bit key in shared memory (bitonic),
// keeping the first m: key = (K - count) << 32 | id for the plain form,
// or (~orderable(score)) << 32 | id for a learned score.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kMaxK = 4096;

__global__ void agree_kernel(const uint32_t* __restrict__ qh, const uint32_t* __restrict__ ph,
                             const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cand,
                             int64_t Q, int64_t cap, int K, int bands, int rows, uint32_t T,
                             uint16_t* __restrict__ count, uint32_t* __restrict__ bandmask,
                             const int* __restrict__ d_flags)
{
    __shared__ uint32_t eqbits[8][kMaxK / 32];  // per warp: equality bit per hash
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (d_flags && *d_flags) return;  // failed validation or candidate overflow
    const int64_t E = min(row_ptr[Q], cap);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; e < E; e += nwarps) {
        // find the query of pair e (binary search over row_ptr)
        int64_t lo = 0, hi = Q;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= e) lo = mid;
            else hi = mid;
        }
        const uint32_t* a = qh + lo * K;
        const uint32_t* b = ph + (int64_t)cand[e] * K;
        int c = 0;
        if ((K & 3) == 0) {
            const uint4* a4 = reinterpret_cast<const uint4*>(a);
            const uint4* b4 = reinterpret_cast<const uint4*>(b);
            for (int base = 0; base < K / 4; base += 32) {
                int i = base + lane;
                unsigned bits = 0;
                if (i < K / 4) {
                    uint4 x = __ldg(a4 + i), y = __ldg(b4 + i);
                    bits = (unsigned)((x.x == y.x) & (x.x != T)) |
                           ((unsigned)((x.y == y.y) & (x.y != T)) << 1) |
                           ((unsigned)((x.z == y.z) & (x.z != T)) << 2) |
                           ((unsigned)((x.w == y.w) & (x.w != T)) << 3);
                }
                c += __popc(bits);
                // hash 4*i + t is bit (4*i + t) % 32 of word (4*i + t) / 32 = i / 8 of the
                // equality mask: OR the nibbles of each group of eight lanes together
                unsigned w0 = bits << ((lane & 7) * 4);
                w0 |= __shfl_xor_sync(0xffffffffu, w0, 1);
                w0 |= __shfl_xor_sync(0xffffffffu, w0, 2);
                w0 |= __shfl_xor_sync(0xffffffffu, w0, 4);
                if ((lane & 7) == 0 && i < K / 4) eqbits[wid][i >> 3] = w0;
            }
        } else {
            for (int base = 0; base < K; base += 32) {
                int i = base + lane;
                bool eq = i < K && a[i] == b[i] && a[i] != T;
                unsigned bal = __ballot_sync(0xffffffffu, eq);
                c += eq;
                if (lane == 0) eqbits[wid][base / 32] = bal;
            }
        }
        __syncwarp();
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) count[e] = (uint16_t)c;
        if (bandmask) {
            unsigned ok = 0;
            for (int j = lane; j < bands && j < 32; j += 32) {
                bool all = true;
                for (int t = 0; t < rows; ++t) {
                    int k = j * rows + t;
                    all &= (eqbits[wid][k >> 5] >> (k & 31)) & 1u;
                }
                ok = all;
            }
            unsigned m = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) bandmask[e] = m;
        }
        __syncwarp();
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
        for (int i = threadIdx.x; i < cap; i += blockDim.x) {
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
        bitonic_sort_u64(s, cap);
        kept = min(m, kept + take);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        out_ids[q * m + i] = i < kept ? (int32_t)(uint32_t)(s[i] & 0xFFFFFFFFu) : -1;
    if (threadIdx.x == 0) out_n[q] = kept;
}

}  // namespace

int pmh_launch_agree(pmh_ctx ctx, const uint32_t* qh, const uint32_t* ph, const int64_t* row_ptr,
                     const int32_t* cand, int64_t Q, int64_t cap, const pmh_params* P,
                     uint16_t* count, uint32_t* bandmask, const int* d_flags, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    int blocks = ctx->sm_count * 8;
    agree_kernel<<<blocks, 256, 0, s>>>(qh, ph, row_ptr, cand, Q, cap, (int)P->K, (int)P->bands,
                                        (int)P->rows, P->T, count, bandmask, d_flags);
    PMH_LAUNCHED("agree_kernel");
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

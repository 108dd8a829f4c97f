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
constexpr int kAgreeChunk = 64;  // consecutive pairs per warp turn
constexpr int kAgreeGroup = 4;   // pairs compared at a time (their loads in flight together)

// Warps take chunks of kAgreeChunk consecutive pairs (the row of the first by
// binary search over row_ptr); 32 pairs at a time each lane reads one pair's
// candidate id and steps its row on from there, and the warp then compares the
// pairs four at a time (ids and rows by shuffle).  Per pair:
// equality bits of the K hashes (16-byte loads when K % 4 == 0), the count (warp
// sum), the full-match bits of the first 32 bands and, optionally, the reranker's
// feature row.
template <bool kFeat>  // feature rows written (a build without their work for the counts alone)
__global__ void __launch_bounds__(kAgreeWarps * 32, 6)
agree_rows_kernel(const uint32_t* __restrict__ qh, const uint32_t* __restrict__ ph,
                  const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cand, int64_t Q,
                  int64_t cap, int K, int bands, int rows, uint32_t T, uint16_t* __restrict__ count,
                  uint32_t* __restrict__ bandmask, __nv_bfloat16* __restrict__ feat, FeatSrc qf,
                  FeatSrc pf, const int* __restrict__ d_flags)
{
    __shared__ uint32_t eqbits[kAgreeWarps][kAgreeGroup][kMaxK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (d_flags && *d_flags) return;  // failed validation or candidate overflow
    const int64_t total = min(row_ptr[Q], cap);
    const int64_t nwarps = (int64_t)gridDim.x * kAgreeWarps;
    const int K4 = K / 4;
    // equality words in shared memory: for the band bits, and for the features' groups
    // unless K = 128 (then lane l holds group l's four hashes)
    const bool need_eq = bandmask || (kFeat && K != 128);
    for (int64_t ch = (int64_t)blockIdx.x * kAgreeWarps + wid; ch * kAgreeChunk < total; ch += nwarps) {
        const int64_t x0 = ch * kAgreeChunk, x1 = min(x0 + kAgreeChunk, total);
        // the row holding pair x0: the last q with row_ptr[q] <= x0
        int64_t lo = 0, hi = Q;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= x0) lo = mid;
            else hi = mid;
        }
        const int64_t q0 = lo;
        for (int64_t xb = x0; xb < x1; xb += 32) {
            const int nvalid = (int)min((int64_t)32, x1 - xb);
            const int64_t xl = xb + lane;
            int64_t ql = q0;
            int32_t pl = 0;
            if (lane < nvalid) {
                while (row_ptr[ql + 1] <= xl) ++ql;
                pl = cand[xl];
            }
            for (int t0 = 0; t0 < nvalid; t0 += kAgreeGroup) {
                const int64_t x = xb + t0;
                int64_t qq[kAgreeGroup], pp[kAgreeGroup];
                bool ok[kAgreeGroup];
    #pragma unroll
                for (int t = 0; t < kAgreeGroup; ++t) {
                    ok[t] = t0 + t < nvalid;
                    qq[t] = __shfl_sync(0xffffffffu, ql, (t0 + t) & 31);
                    pp[t] = __shfl_sync(0xffffffffu, pl, (t0 + t) & 31);
                }
                // lt / gt: hashes with h(q) < h(p) / h(q) > h(p); grp: K = 128, lane l's four
                // hashes (group l of the features' 32-group split) all equal
                int c[kAgreeGroup] = {0, 0, 0, 0}, lt[kAgreeGroup] = {0, 0, 0, 0}, gt[kAgreeGroup] = {0, 0, 0, 0};
                bool grp[kAgreeGroup] = {false, false, false, false};
                if ((K & 3) == 0) {
                    for (int base = 0; base < K4; base += 32) {
                        const int i = base + lane;
                        uint4 u[kAgreeGroup], v[kAgreeGroup];
    #pragma unroll
                        for (int t = 0; t < kAgreeGroup; ++t) {
                            u[t] = v[t] = make_uint4(0u, 0u, 0u, 0u);
                            if (ok[t] && i < K4) {
                                u[t] = __ldg(reinterpret_cast<const uint4*>(qh + qq[t] * K) + i);
                                v[t] = __ldg(reinterpret_cast<const uint4*>(ph + pp[t] * K) + i);
                            }
                        }
    #pragma unroll
                        for (int t = 0; t < kAgreeGroup; ++t) {
                            unsigned bits = 0;
                            if (i < K4) {
                                bits = (unsigned)((u[t].x == v[t].x) & (u[t].x != T)) |
                                       ((unsigned)((u[t].y == v[t].y) & (u[t].y != T)) << 1) |
                                       ((unsigned)((u[t].z == v[t].z) & (u[t].z != T)) << 2) |
                                       ((unsigned)((u[t].w == v[t].w) & (u[t].w != T)) << 3);
                                if (kFeat) {
                                    lt[t] += (u[t].x < v[t].x) + (u[t].y < v[t].y) + (u[t].z < v[t].z) +
                                             (u[t].w < v[t].w);
                                    gt[t] += (u[t].x > v[t].x) + (u[t].y > v[t].y) + (u[t].z > v[t].z) +
                                             (u[t].w > v[t].w);
                                }
                            }
                            c[t] += __popc(bits);
                            grp[t] = bits == 0xFu;
                            if (need_eq) {
                                // hash 4i+e is bit (4i+e) % 32 of word i / 8: OR eight lanes' nibbles
                                unsigned w0 = bits << ((lane & 7) * 4);
                                w0 |= __shfl_xor_sync(0xffffffffu, w0, 1);
                                w0 |= __shfl_xor_sync(0xffffffffu, w0, 2);
                                w0 |= __shfl_xor_sync(0xffffffffu, w0, 4);
                                if ((lane & 7) == 0 && i < K4) eqbits[wid][t][i >> 3] = w0;
                            }
                        }
                    }
                } else {
                    for (int base = 0; base < K; base += 32) {
                        const int i = base + lane;
    #pragma unroll
                        for (int t = 0; t < kAgreeGroup; ++t) {
                            const bool in = ok[t] && i < K;
                            const uint32_t a = in ? qh[qq[t] * K + i] : 0u, b = in ? ph[pp[t] * K + i] : 0u;
                            const bool eq = in && a == b && a != T;
                            const unsigned bal = __ballot_sync(0xffffffffu, eq);
                            c[t] += eq;
                            if (kFeat && in) {
                                lt[t] += a < b;
                                gt[t] += a > b;
                            }
                            if (lane == 0) eqbits[wid][t][base / 32] = bal;
                        }
                    }
                }
                __syncwarp();
    #pragma unroll
                for (int t = 0; t < kAgreeGroup; ++t) {
                    if (!ok[t]) continue;  // warp-uniform
                    const int64_t xt = x + t;
                    int ct, ltt = 0, gtt = 0;
                    if (kFeat && K < 1024) {  // the three counts in one sum (10 bits each)
                        const int sum = __reduce_add_sync(0xffffffffu, c[t] | (lt[t] << 10) | (gt[t] << 20));
                        ct = sum & 1023;
                        ltt = (sum >> 10) & 1023;
                        gtt = sum >> 20;
                    } else {
                        ct = __reduce_add_sync(0xffffffffu, c[t]);
                        if (kFeat) {
                            ltt = __reduce_add_sync(0xffffffffu, lt[t]);
                            gtt = __reduce_add_sync(0xffffffffu, gt[t]);
                        }
                    }
                    if (count && lane == 0) count[xt] = (uint16_t)ct;
                    if (bandmask) {
                        bool all = lane < bands;
                        for (int r = 0; r < rows && all; ++r) {
                            const int k = lane * rows + r;
                            all = (eqbits[wid][t][k >> 5] >> (k & 31)) & 1u;
                        }
                        const unsigned mb = __ballot_sync(0xffffffffu, all);
                        if (lane == 0) bandmask[xt] = mb;
                    }
                    if (kFeat) {
                        float flo, fhi;
                        if (K == 128) {
                            flo = grp[t] ? 1.f : 0.f;
                            fhi = pmh_feature_col(lane, K, ct, ltt, gtt, pmh_feat_pair(qf, pf, qq[t], pp[t]));
                        } else {
                            pmh_feature_values(eqbits[wid][t], K, ct, ltt, gtt, pmh_feat_pair(qf, pf, qq[t], pp[t]),
                                               lane, flo, fhi);
                        }
                        __nv_bfloat16* f = feat + xt * 48;
                        f[lane] = __float2bfloat16_rn(flo);
                        if (lane < 16) f[32 + lane] = __float2bfloat16_rn(fhi);
                    }
                }
                __syncwarp();
            }
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

// one block per query.  Count form: a histogram of the row's counts (0..K) gives
// the largest threshold c* with at least m pairs of count >= c*; every key of
// those pairs is gathered and sorted, and the first m kept -- the m best keys
// (count desc, id asc) all have count >= c*, so the list is the full sort's.  A
// row whose gathered set would pass kSelMax (a long tie at c*), and the score
// form, take the merge form: the running top-m kept in s[0..m), each new chunk
// of the row appended and sorted with it.
constexpr int kSelMax = 2048;

__global__ void __launch_bounds__(kTopThreads)
topm_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cand,
            const uint16_t* __restrict__ count, const float* __restrict__ score, int K, int m,
            int cap /* power of two >= max(m + kTopChunk, kSelMax) */, int32_t* __restrict__ out_ids,
            int32_t* __restrict__ out_n, const int* __restrict__ d_flags)
{
    extern __shared__ uint64_t s[];  // cap keys, then (count form) K + 1 histogram bins
    __shared__ int sel_c, sel_total, sel_n;
    const int64_t q = blockIdx.x;
    const bool failed = d_flags && *d_flags;
    const int64_t b = failed ? 0 : row_ptr[q], e = failed ? 0 : row_ptr[q + 1];
    int kept = 0;
    bool merged = true;
    if (!score && e - b > m) {
        int* hist = reinterpret_cast<int*>(s + cap);
        for (int i = threadIdx.x; i <= K; i += blockDim.x) hist[i] = 0;
        if (threadIdx.x == 0) {  // (the warp below always finds the threshold)
            sel_c = 0;
            sel_total = (int)min(e - b, (int64_t)INT32_MAX);
            sel_n = 0;
        }
        __syncthreads();
        for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x) atomicAdd(&hist[min((int)count[x], K)], 1);
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane l sums bins [l*seg, (l+1)*seg); suffix sums over the lanes find the
            // lane holding c*, which then walks its bins downwards
            const int lane = threadIdx.x, seg = (K + 32) / 32;
            const int lo = lane * seg, hi = min(lo + seg, K + 1);
            int mine = 0;
            for (int c = lo; c < hi; ++c) mine += hist[c];
            int suf = mine;  // bins >= lo
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_down_sync(0xffffffffu, suf, o);
                if (lane + o < 32) suf += y;
            }
            const int above = suf - mine;  // bins >= hi
            if (above < m && suf >= m) {
                int acc = above, c = hi - 1;
                for (; c >= lo; --c) {
                    acc += hist[c];
                    if (acc >= m) break;
                }
                sel_c = c;
                sel_total = acc;
            }
        }
        __syncthreads();
        const int cstar = sel_c, total = sel_total;
        if (total <= kSelMax) {
            merged = false;
            for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x) {
                const int c = min((int)count[x], K);
                if (c >= cstar) {
                    const int pos = atomicAdd(&sel_n, 1);
                    if (pos < total) s[pos] = ((uint64_t)(uint32_t)(K - c) << 32) | (uint32_t)cand[x];
                }
            }
            int sz = 2;
            while (sz < total) sz <<= 1;
            for (int i = total + threadIdx.x; i < sz; i += blockDim.x) s[i] = ~0ull;
            __syncthreads();
            bitonic_sort_u64(s, sz);
            kept = m;
        }
    }
    for (int64_t base = b; merged && base < e; base += kTopChunk) {
        int take = (int)(e - base < kTopChunk ? e - base : kTopChunk);
        // sort only the occupied prefix, rounded up to a power of two (most lists are short)
        int sz = 2;
        while (sz < kept + take) sz <<= 1;
        for (int i = threadIdx.x; i < sz; i += blockDim.x) {
            uint64_t key = ~0ull;
            if (i >= kept && i < kept + take) {
                int64_t idx = base + (i - kept);
                uint32_t hi = score ? ~f2ord(score[idx]) : (uint32_t)(K - min((int)count[idx], K));
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
    auto fn = feat ? agree_rows_kernel<true> : agree_rows_kernel<false>;
    fn<<<blocks, kAgreeWarps * 32, 0, s>>>(qh, ph, row_ptr, cand, Q, cap, (int)P->K, (int)P->bands, (int)P->rows,
                                           P->T, count, bandmask, reinterpret_cast<__nv_bfloat16*>(feat), qf,
                                           pf, d_flags);
    PMH_LAUNCHED("agree_rows_kernel");
    return PMH_OK;
}

int pmh_launch_topm(const int64_t* row_ptr, const int32_t* cand, const uint16_t* count,
                    const float* score, int64_t Q, int32_t m, int K, int32_t* out_ids, int32_t* out_n,
                    const int* d_flags, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    int cap = 1;
    while (cap < m + kTopChunk || cap < kSelMax) cap <<= 1;
    const int kb = (K > 0 && K <= kMaxK) ? K : kMaxK;  // counts are <= K
    const size_t smem = sizeof(uint64_t) * cap + sizeof(int) * (size_t)(kb + 1);
    PMH_CUDA_TRY(cudaFuncSetAttribute(topm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    topm_kernel<<<(unsigned)Q, kTopThreads, smem, s>>>(row_ptr, cand, count, score, kb, m, cap,
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
    return pmh_launch_topm(d_row_ptr, d_cand, d_count, d_score, Q, m, 0, d_out_ids, d_out_n, nullptr,
                           (cudaStream_t)stream);
}

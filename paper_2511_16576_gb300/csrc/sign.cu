// sign.cu -- step A1: MinHash signatures (Definition 2, Algorithm 1).
//
// h_k(P) = min{ i in [0,T) : point i of stream k lies in P }, else T.
//
// GB300 mapping.  The work is pure 32/64-bit integer arithmetic: the point
// generator (two 64-bit multiplies per point) dominates, the bbox test rejects
// almost every point, and the exact point-in-polygon test runs ~2-3 times per
// hash.  One warp owns a work item (polygon p, 32 consecutive hashes):
//   * the polygon's vertices are staged once into the warp's shared-memory
//     slice and its edges binned into 32 horizontal slabs there, so that an
//     exact test reads only the few edges whose y-range meets the point's slab
//     (polygons of more than 256 vertices are read from global memory through
//     their y-slab edge index instead, see slabs.cu);
//   * per round every lane draws U points (indices i0 + j*32 + lane), so one
//     round covers 32*U consecutive stream indices; the counter-based stream
//     lets each lane jump straight to its own index;
//   * lanes whose point passes the half-open bbox test are visited in index
//     order (ballot + ffs); each candidate is tested by the whole warp, lanes
//     splitting the edges, parity by ballot/popc -- the first inside point is
//     the hash, exactly the min of the definition;
//   * lane j keeps the hash of k0 + j and the warp writes 32 hashes with one
//     coalesced store.
// Items are handed out by a global atomic ticket (persistent grid sized to the
// SM count) in decreasing order of expected cost (2^32 / area per hash,
// Theorem 2: E[h] = 1/S_p), which balances polygons whose work differs by
// orders of magnitude.
//
// Which kernel signs which polygon: with the stream index, every polygon is
// signed by one launch of sign_unified_kernel (sign_unified.cu: indexed or walk
// form as each polygon's plan says, staged or through its y-slab lists); this
// file's sign_kernel signs without the stream index, with precomputed coverage
// masks, and the batches of the captured query pipeline.
#include <algorithm>
#include <mutex>

#include "pmh_internal.cuh"

#include "sign_common.cuh"

namespace {

constexpr int kWarps = 8;        // warps per block
constexpr int kU = 4;            // points per lane per round
constexpr int kWorkSlot = 8;     // context ticket slots 8..13: work counters of the walk kernel
constexpr int kIdxWorkSlot = 16; // slots 16..21: work counters of the unified kernel

__device__ __forceinline__ uint32_t sign_one(const int2* __restrict__ v, int n, int x0, int y0,
                                             uint32_t w, uint32_t h, uint64_t sk, uint32_t T,
                                             int lane)
{
    Work unused;
    return sign_one_t<kU>(AllEdges{v, n}, x0, y0, w, h, sk, T, lane, unused);
}

// Indexed form: the stream points of index < lim that fall in the bounding box
// are read from the cells under it (kCand per hash at most, else the full walk).
constexpr int kCand = 64;

// Indexed form of the hashes k0 .. kend-1, four at a time: each group of eight
// lanes gathers one hash's candidates from the cells under the bounding box
// (four independent chains of index reads in flight per warp), then the warp
// resolves the four hashes one after the other: candidates in index order by
// repeated warp argmin, exact test, walk resumed at lim if none is inside.
template <int U, class Inside>
__device__ uint32_t sign_chunk_indexed(const Inside& inside, const StreamIndexView& S, int4 bb,
                                       uint64_t seed, int k0, int kend, uint32_t T, uint32_t lim,
                                       uint2* cbuf /* [4][kCand] */, int* ccount /* [4] */,
                                       int lane, Work& work)
{
    const uint32_t w = (uint32_t)(bb.z - bb.x), h = (uint32_t)(bb.w - bb.y);
    lim = min(lim, T);
    const int cx0 = bb.x >> S.shift, cx1 = (bb.z - 1) >> S.shift;
    const int cy0 = bb.y >> S.shift, cy1 = (bb.w - 1) >> S.shift;
    const int ncx = cx1 - cx0 + 1, C = ncx * (cy1 - cy0 + 1);
    const int g = lane >> 3, gl = lane & 7;
    uint32_t mine = T;
    for (int kb = k0; kb < kend; kb += 4) {
        if (lane < 4) ccount[lane] = 0;
        __syncwarp();
        const int k = kb + g;
        int read = 0;
        if (k < kend) {
            const uint2* cs = S.cell + k;  // record of cell c: cs[c * K]
            uint2* cb = cbuf + g * kCand;
            for (int c = gl; c < C; c += 8) {
                const int cell = ((cy0 + c / ncx) << S.gbits) | (cx0 + c % ncx);
                const uint32_t beg = cs[(int64_t)cell * S.K].x, end = cs[(int64_t)(cell + 1) * S.K].x;
                for (uint32_t e = beg; e < end; e += 4) {
                    uint2 q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        q[u] = e + u < end ? S.ent[e + u] : make_uint2(0xFFFFFFFFu, 0u);
                    bool stop = false;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (stop || e + u >= end) break;
                        ++read;
                        if (q[u].x >= lim) {
                            stop = true;
                            break;
                        }
                        const uint32_t r = q[u].y;
                        if (((r & 0xFFFFu) - (uint32_t)bb.x) < w && ((r >> 16) - (uint32_t)bb.y) < h) {
                            const int slot = atomicAdd(&ccount[g], 1);
                            if (slot < kCand) cb[slot] = make_uint2(q[u].x, r);
                        }
                    }
                    if (stop) break;
                }
            }
        }
        work.entries += __reduce_add_sync(0xffffffffu, read);
        __syncwarp();
        const int nk = min(4, kend - kb);
        work.cells += (unsigned long long)C * nk;
        for (int j = 0; j < nk; ++j) {
            const int kk = kb + j;
            const int n = ccount[j];
            const uint64_t sk = pmh_mix64(seed + (uint64_t)(kk + 1) * PMH_GAMMA);
            uint32_t hk = 0xFFFFFFFFu;
            work.cand += min(n, kCand);
            if (n > kCand) {
                hk = sign_resume<U>(inside, bb.x, bb.y, w, h, sk, T, lane, &work, 0);
            } else {
                const uint2* cb = cbuf + j * kCand;
                uint2 c0 = lane < n ? cb[lane] : make_uint2(0xFFFFFFFFu, 0u);
                uint2 c1 = lane + 32 < n ? cb[lane + 32] : make_uint2(0xFFFFFFFFu, 0u);
                for (int t = 0; t < n; ++t) {
                    const uint32_t best = __reduce_min_sync(0xffffffffu, min(c0.x, c1.x));
                    const unsigned who = __ballot_sync(0xffffffffu, c0.x == best || c1.x == best);
                    const int src = __ffs(who) - 1;
                    const uint32_t r = __shfl_sync(0xffffffffu, c0.x == best ? c0.y : c1.y, src);
                    if (inside((int)(r & 0xFFFFu), (int)(r >> 16), lane, work)) {
                        hk = best;
                        break;
                    }
                    if (lane == src) {
                        if (c0.x == best) c0.x = 0xFFFFFFFFu;
                        else c1.x = 0xFFFFFFFFu;
                    }
                }
                if (hk == 0xFFFFFFFFu)
                    hk = lim >= T ? T : sign_resume<U>(inside, bb.x, bb.y, w, h, sk, T, lane, &work, lim);
            }
            if (lane == kk - k0) mine = hk;
        }
        __syncwarp();
    }
    return mine;
}

// the hashes k0 .. k0+31 of one polygon; lane j returns hash k0 + j.  lim > 0
// selects the indexed form (stream points below lim read from the index).
template <int U, class Inside>
__device__ __forceinline__ uint32_t sign_chunk_walk(const Inside& inside, int4 bb, uint64_t seed,
                                                    int k0, int kend, uint32_t T, int lane, Work& work)
{
    const uint32_t w = (uint32_t)(bb.z - bb.x), h = (uint32_t)(bb.w - bb.y);
    uint32_t mine = T;
    for (int k = k0; k < kend; ++k) {
        uint64_t sk = pmh_mix64(seed + (uint64_t)(k + 1) * PMH_GAMMA);
        uint32_t hk = sign_one_t<U>(inside, bb.x, bb.y, w, h, sk, T, lane, work);
        if (lane == k - k0) mine = hk;
    }
    return mine;
}

template <int U, class Inside>
__device__ __forceinline__ uint32_t sign_chunk(const Inside& inside, int4 bb, uint64_t seed, int k0,
                                               int kend, uint32_t T, int lane,
                                               const StreamIndexView& S, uint32_t lim,
                                               uint2* cbuf, int* ccount, Work& work)
{
    if (lim) return sign_chunk_indexed<U>(inside, S, bb, seed, k0, kend, T, lim, cbuf, ccount, lane, work);
    return sign_chunk_walk<U>(inside, bb, seed, k0, kend, T, lane, work);
}


template <int U, int W, int MinBlocks>
__global__ void __launch_bounds__(W * 32, MinBlocks)
sign_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
            const int4* __restrict__ bbox, const SlabInfo* __restrict__ slabs,
            const int32_t* __restrict__ slab_ptr, const int32_t* __restrict__ slab_edges,
            const int32_t* __restrict__ order, uint64_t seed, int K, uint32_t T, int chunks,
            int64_t n_polys, const int64_t* __restrict__ d_n, const int* __restrict__ d_flags,
            unsigned long long* __restrict__ ticket, uint32_t* __restrict__ out,
            const int64_t* __restrict__ area2, StreamIndexView S,
            unsigned long long* __restrict__ work_out, const uint32_t* __restrict__ masks)
{
    __shared__ __align__(16) int2 sv[W][kSmemVerts + 1];
    __shared__ uint8_t sid[W][kSlabCap];
    __shared__ uint16_t sbeg[W][kSlabs + 1];
    __shared__ int scnt[W][kSlabs];
    __shared__ uint2 cbuf[W][4 * kCand];
    __shared__ int ccount[W][4];
    __shared__ uint32_t smask[W][16];
    __shared__ unsigned long long wsum[6];
    Work work;
    if (threadIdx.x < 6) wsum[threadIdx.x] = 0;
    __syncthreads();
    if (d_flags && *d_flags) return;  // the batch failed validation
    if (d_n) n_polys = min(n_polys, *d_n);
    const int64_t n_items = n_polys * chunks;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(ticket, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= n_items) break;
        const int64_t slot = (int64_t)(item / (unsigned)chunks);
        const int64_t p = order ? (int64_t)order[slot] : slot;
        const int k0 = (int)(item % (unsigned)chunks) * 32;
        const int kend = min(K, k0 + 32);
        const int64_t b = off[p];
        const int n = (int)(off[p + 1] - b);
        const int4 bb = bbox[p];
        // (with the stream index every polygon is signed by sign_unified.cu instead)
        const uint32_t lim = area2 && S.cell && n > kSmemVerts ? pmh_indexed_limit(bb, area2[p]) : 0;
        uint32_t mine;
        if (n <= kSmemVerts) {
            // stage the vertices (closed: v[n] = v[0]; cp.async 8-byte copies), the
            // coverage mask if any, and the slab lists in this warp's shared-memory slice
            if (masks && lane < 16) smask[wid][lane] = masks[p * 16 + lane];
            stage_vertices(sv[wid], xy + b, n, lane);
            const int sh = staged_slab_shift(max(bb.w - bb.y, 1));
            const bool staged = bb.w > bb.y && bb.z > bb.x &&
                                build_staged_slabs(sv[wid], n, bb.y, sh, sid[wid], sbeg[wid], scnt[wid], lane);
            const int cwl = mask_cell_log2(bb.z - bb.x), chl = mask_cell_log2(bb.w - bb.y);
            if (staged) {
                const StagedEdges st{sv[wid], sid[wid], sbeg[wid], bb.y, sh};
                if (masks)
                    mine = sign_chunk_walk<U>(Masked<StagedEdges>{st, smask[wid], bb.x, bb.y, cwl, chl}, bb,
                                              seed, k0, kend, T, lane, work);
                else
                    mine = sign_chunk_walk<U>(st, bb, seed, k0, kend, T, lane, work);
            } else {
                // too many slab references (or an empty box): every edge, no mask
                mine = sign_chunk_walk<U>(AllEdges{sv[wid], n}, bb, seed, k0, kend, T, lane, work);
            }
        } else if (slabs && slabs[p].S > 0) {
            const SlabInfo si = slabs[p];
            mine = sign_chunk<U>(SlabEdges{xy + b, n, slab_ptr + si.slab_base,
                                           slab_edges + si.edge_base, si.slab_h, si.ymin},
                                 bb, seed, k0, kend, T, lane, S, lim, cbuf[wid], ccount[wid], work);
        } else {
            mine = sign_chunk<U>(AllEdges{xy + b, n}, bb, seed, k0, kend, T, lane, S, lim,
                                 cbuf[wid], ccount[wid], work);
        }
        if (k0 + lane < kend) out[p * (int64_t)K + k0 + lane] = mine;
        __syncwarp();
    }
    if (work_out) {
        unsigned long long le = work.lane_edges;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) le += __shfl_xor_sync(0xffffffffu, le, o);
        work.edges += le;
        if (lane == 0) {
            atomicAdd(&wsum[0], work.walk);
            atomicAdd(&wsum[1], work.cells);
            atomicAdd(&wsum[2], work.entries);
            atomicAdd(&wsum[3], work.cand);
            atomicAdd(&wsum[4], work.edges);
            atomicAdd(&wsum[5], work.masked);
        }
        __syncthreads();
        if (threadIdx.x < 6) atomicAdd(&work_out[threadIdx.x], wsum[threadIdx.x]);
    }
}

using SignFn = void (*)(const int2*, const int64_t*, const int4*, const SlabInfo*, const int32_t*,
                        const int32_t*, const int32_t*, uint64_t, int, uint32_t, int, int64_t,
                        const int64_t*, const int*, unsigned long long*, uint32_t*, const int64_t*,
                        StreamIndexView, unsigned long long*, const uint32_t*);
struct SignVariant {
    int U, W, MinBlocks;
    SignFn fn;
};
// index 0 is the default; the autotuner may pick any of them.  MinBlocks caps
// the registers (65536 / (MinBlocks * W * 32)) so that more warps stay resident
// to hide the latency of the index reads.  (Static shared memory per block
// stays below 48 KiB: 8 warps at most.)
const SignVariant kSignVariants[] = {
    {4, 8, 3, sign_kernel<4, 8, 3>}, {4, 8, 4, sign_kernel<4, 8, 4>}, {4, 8, 2, sign_kernel<4, 8, 2>},
    {2, 8, 3, sign_kernel<2, 8, 3>}, {2, 8, 4, sign_kernel<2, 8, 4>}, {8, 8, 3, sign_kernel<8, 8, 3>},
};
constexpr int kNumSignVariants = sizeof(kSignVariants) / sizeof(kSignVariants[0]);

}  // namespace

int pmh_sign_variant_count() { return kNumSignVariants; }

void pmh_sign_variant_shape(int v, int* points_per_lane, int* warps)
{
    *points_per_lane = kSignVariants[v].U;
    *warps = kSignVariants[v].W;
}

int pmh_launch_sign(pmh_ctx ctx, const int2* xy, const int64_t* off, const int4* bbox,
                    const SlabInfo* slabs, const int32_t* slab_ptr, const int32_t* slab_edges,
                    const int32_t* order, const pmh_params* P, int64_t n_polys,
                    const int64_t* d_n, const int* d_flags, unsigned long long* ticket,
                    uint32_t* out, cudaStream_t s, const int64_t* area2,
                    const StreamIndexView* sidx, const uint32_t* masks,
                    const int32_t* order_cls, int64_t n_indexed, int64_t n_whole_cost)
{
    const StreamIndexView S = sidx ? *sidx : StreamIndexView{};
    if (n_polys <= 0) return PMH_OK;
    unsigned long long* work = d_n ? nullptr : ctx->d_tickets + kWorkSlot;
    if (work) {
        PMH_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(unsigned long long) * 6, s));
        PMH_CUDA_TRY(cudaMemsetAsync(ctx->d_tickets + kIdxWorkSlot, 0, sizeof(unsigned long long) * 6, s));
        if (!ctx->sign_count) work = nullptr;  // counts stay zero: the counter-free kernels run
    }
    const bool timed = ctx->sign_timing && !d_n && ctx->sign_ev_used + 3 <= 3 * 1024;
    cudaEvent_t* ev = nullptr;
    if (timed) {
        while (ctx->sign_ev.size() < ctx->sign_ev_used + 3) {
            cudaEvent_t e;
            PMH_CUDA_TRY(cudaEventCreate(&e));
            ctx->sign_ev.push_back(e);
        }
        ev = ctx->sign_ev.data() + ctx->sign_ev_used;
        ctx->sign_ev_used += 3;
        PMH_CUDA_TRY(cudaEventRecord(ev[0], s));
    }
    if (S.cell && S.ranked && order_cls && area2 && !d_n && !masks) {
        // every polygon in one launch: the class order puts the polygons above
        // kChunkMinVerts first (32-hash items), then the rest (whole polygons)
        const int U = kSignVariants[ctx->sign_variant >= 0 ? ctx->sign_variant : 0].U;
        const int64_t n_big = n_polys - n_indexed - n_whole_cost;
        PMH_TRY(pmh_launch_sign_unified(ctx, U, xy, off, bbox, area2, slabs, slab_ptr, slab_edges,
                                        order_cls, n_polys, n_big, n_indexed, nullptr, nullptr, P, S,
                                        ticket + 2, out, work ? ctx->d_tickets + kIdxWorkSlot : nullptr, s));
        if (timed) {
            PMH_CUDA_TRY(cudaEventRecord(ev[1], s));
            PMH_CUDA_TRY(cudaEventRecord(ev[2], s));
        }
        return PMH_OK;
    }
    if (timed) PMH_CUDA_TRY(cudaEventRecord(ev[1], s));
    if (n_polys <= 0) {
        if (timed) PMH_CUDA_TRY(cudaEventRecord(ev[2], s));
        return PMH_OK;
    }
    const SignVariant& v = kSignVariants[ctx->sign_variant >= 0 ? ctx->sign_variant : 0];
    const int chunks = (int)((P->K + 31) / 32);
    const int64_t n_items = n_polys * chunks;
    int per_sm = 0;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, v.W * 32, 0));
    int64_t blocks = (int64_t)ctx->sm_count * std::max(per_sm, 1);
    blocks = std::min<int64_t>(blocks, (n_items + v.W - 1) / v.W);
    PMH_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    v.fn<<<(int)blocks, v.W * 32, 0, s>>>(xy, off, bbox, slabs, slab_ptr, slab_edges, order,
                                          P->seed, (int)P->K, P->T, chunks, n_polys, d_n, d_flags,
                                          ticket, out, area2, S, work, masks);
    PMH_LAUNCHED("sign_kernel");
    if (timed) PMH_CUDA_TRY(cudaEventRecord(ev[2], s));
    return PMH_OK;
}

extern "C" int pmh_minhash_sign(pmh_ctx ctx, pmh_polys polys, const pmh_params* params,
                                uint32_t* d_hashes, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (!polys || (!d_hashes && polys->n > 0))
        return pmh_set_error(PMH_ERR_ARG, "null polygons or output");
    if (polys->n == 0) return PMH_OK;
    StreamIndexView sidx;
    const bool indexed = (params->flags & PMH_FLAG_STREAM_INDEX) != 0;
    const bool masked = (params->flags & PMH_FLAG_COVERAGE_MASK) != 0;
    if (indexed) PMH_TRY(pmh_stream_index_get(ctx, params, (cudaStream_t)stream, &sidx));
    if ((!indexed || !sidx.ranked || masked) && !polys->order)
        PMH_TRY(pmh_build_cost_order(polys, (cudaStream_t)stream));
    if (masked && !polys->mask) PMH_TRY(pmh_build_masks(polys, (cudaStream_t)stream));
    return pmh_launch_sign(ctx, polys->xy, polys->offsets, polys->bbox, polys->slab_info,
                           polys->slab_ptr, polys->slab_edges, polys->order, params, polys->n,
                           nullptr, nullptr, ctx->d_tickets + 0, d_hashes, (cudaStream_t)stream,
                           polys->area2, indexed ? &sidx : nullptr, masked ? polys->mask : nullptr,
                           polys->order_cls, polys->n_indexed, polys->n_whole_cost);
}

extern "C" int pmh_sign_work(pmh_ctx ctx, uint64_t* h_counts)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!h_counts) return pmh_set_error(PMH_ERR_ARG, "null output");
    uint64_t both[12];
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    PMH_CUDA_TRY(cudaMemcpy(both, ctx->d_tickets + kIdxWorkSlot, sizeof(uint64_t) * 6,
                            cudaMemcpyDeviceToHost));
    PMH_CUDA_TRY(cudaMemcpy(both + 6, ctx->d_tickets + kWorkSlot, sizeof(uint64_t) * 6,
                            cudaMemcpyDeviceToHost));
    for (int i = 0; i < 6; ++i) h_counts[i] = both[i] + both[6 + i];
    return PMH_OK;
}

extern "C" int pmh_sign_count_work(pmh_ctx ctx, int enable)
{
    if (!ctx) return pmh_set_error(PMH_ERR_ARG, "null context");
    ctx->sign_count = enable != 0;
    return PMH_OK;
}

extern "C" int pmh_sign_timing(pmh_ctx ctx, int enable)
{
    if (!ctx) return pmh_set_error(PMH_ERR_ARG, "null context");
    ctx->sign_timing = enable != 0;
    return PMH_OK;
}

extern "C" int pmh_sign_report(pmh_ctx ctx, float* h_ms, uint64_t* h_counts)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    if (h_ms) {
        double a = 0.0, b = 0.0;
        const size_t calls = ctx->sign_ev_used / 3;
        for (size_t c = 0; c < calls; ++c) {
            float x = 0.0f, y = 0.0f;
            PMH_CUDA_TRY(cudaEventElapsedTime(&x, ctx->sign_ev[3 * c], ctx->sign_ev[3 * c + 1]));
            PMH_CUDA_TRY(cudaEventElapsedTime(&y, ctx->sign_ev[3 * c + 1], ctx->sign_ev[3 * c + 2]));
            a += x;
            b += y;
        }
        h_ms[0] = calls ? (float)(a / calls) : -1.0f;
        h_ms[1] = calls ? (float)(b / calls) : -1.0f;
        h_ms[2] = (float)calls;
        ctx->sign_ev_used = 0;
    }
    if (h_counts) {
        PMH_CUDA_TRY(cudaMemcpy(h_counts, ctx->d_tickets + kIdxWorkSlot, sizeof(uint64_t) * 6,
                                cudaMemcpyDeviceToHost));
        PMH_CUDA_TRY(cudaMemcpy(h_counts + 6, ctx->d_tickets + kWorkSlot, sizeof(uint64_t) * 6,
                                cudaMemcpyDeviceToHost));
    }
    return PMH_OK;
}

extern "C" int pmh_sign_variant_info(int variant, int* points_per_lane, int* warps_per_block)
{
    if (variant < 0 || variant >= kNumSignVariants)
        return pmh_set_error(PMH_ERR_ARG, "variant %d not in [0,%d)", variant, kNumSignVariants);
    if (points_per_lane) *points_per_lane = kSignVariants[variant].U;
    if (warps_per_block) *warps_per_block = kSignVariants[variant].W;
    return PMH_OK;
}

extern "C" int pmh_sign_set_variant(pmh_ctx ctx, int variant)
{
    if (!ctx) return pmh_set_error(PMH_ERR_ARG, "null context");
    if (variant < -1 || variant >= kNumSignVariants)
        return pmh_set_error(PMH_ERR_ARG, "variant %d not in [-1,%d)", variant, kNumSignVariants);
    ctx->sign_variant = variant;
    return PMH_OK;
}

extern "C" int pmh_sign_autotune(pmh_ctx ctx, pmh_polys sample, const pmh_params* params,
                                 int* h_best, float* h_ms)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (!sample || sample->n <= 0 || !h_best)
        return pmh_set_error(PMH_ERR_ARG, "empty sample or null output");
    uint32_t* out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * (size_t)sample->n * params->K) != cudaSuccess) {
        cudaGetLastError();
        return pmh_set_error(PMH_ERR_NOMEM, "autotune output allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved = ctx->sign_variant;
    int best = 0, rc = PMH_OK;
    float best_ms = 1e30f;
    for (int v = 0; v < kNumSignVariants && rc == PMH_OK; ++v) {
        ctx->sign_variant = v;
        float ms_v = 1e30f;
        for (int r = 0; r < 3 && rc == PMH_OK; ++r) {  // first run is a warm-up
            cudaEventRecord(e0, 0);
            StreamIndexView sidx;
            const bool indexed = (params->flags & PMH_FLAG_STREAM_INDEX) != 0;
            const bool masked = (params->flags & PMH_FLAG_COVERAGE_MASK) != 0;
            if (indexed) rc = pmh_stream_index_get(ctx, params, 0, &sidx);
            if (rc == PMH_OK && (!indexed || !sidx.ranked || masked) && !sample->order)
                rc = pmh_build_cost_order(sample, 0);
            if (rc == PMH_OK && masked && !sample->mask) rc = pmh_build_masks(sample, 0);
            if (rc == PMH_OK)
                rc = pmh_launch_sign(ctx, sample->xy, sample->offsets, sample->bbox, sample->slab_info,
                                     sample->slab_ptr, sample->slab_edges, sample->order, params,
                                     sample->n, nullptr, nullptr, ctx->d_tickets + 1, out, 0,
                                     sample->area2, indexed ? &sidx : nullptr,
                                     masked ? sample->mask : nullptr, sample->order_cls,
                                     sample->n_indexed, sample->n_whole_cost);
            cudaEventRecord(e1, 0);
            if (cudaEventSynchronize(e1) != cudaSuccess)
                rc = pmh_set_error(PMH_ERR_CUDA, "autotune run failed");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) ms_v = std::min(ms_v, ms);
        }
        if (h_ms) h_ms[v] = ms_v;
        if (ms_v < best_ms) {
            best_ms = ms_v;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    ctx->sign_variant = rc == PMH_OK ? best : saved;
    *h_best = best;
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the signing entry point.
//
// Some callers cannot let a library call cudaMalloc: a process that reserves
// its whole device-memory budget at start-up, a host whose memory belongs to a
// caching allocator that a side allocation would fragment or starve, or a
// latency-critical loop that cannot absorb the device-wide synchronisation
// cudaFree implies.  For them the scratch this path needs -- the work-queue
// ticket, a validation word and every polygon's bounding box -- lives in one
// file-scope device array, reserved when the library is loaded on a GPU and
// held by every GPU that loads the library until the process exits.
// ---------------------------------------------------------------------------
// element 0: .x/.y = 64-bit work ticket, .z = validation flags; elements 1..:
// clipped bounding boxes of polygons 0 .. PMH_NOALLOC_MAX_POLYS-1 (4 MiB in all)
static __device__ __align__(256) int4 g_sign_scratch[PMH_NOALLOC_MAX_POLYS + 1];

namespace {

__global__ void noalloc_prep_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
                                    int64_t n_polys, int64_t n_vertices, int4* __restrict__ scratch)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int LIM = 1 << 20;
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_polys;
         p += nwarps) {
        int64_t b = off[p], e = off[p + 1];
        int flags = (b < 0 || e > n_vertices || e < b) ? 1 : 0;
        if (e - b < 3) flags |= 2;
        int x0 = 0x7fffffff, y0 = 0x7fffffff, x1 = -0x7fffffff - 1, y1 = -0x7fffffff - 1;
        if (!flags)
            for (int64_t i = b + lane; i < e; i += 32) {
                int2 v = xy[i];
                if (v.x < -LIM || v.x > LIM || v.y < -LIM || v.y > LIM) flags |= 4;
                x0 = min(x0, v.x);
                x1 = max(x1, v.x);
                y0 = min(y0, v.y);
                y1 = max(y1, v.y);
            }
        x0 = __reduce_min_sync(0xffffffffu, x0);
        y0 = __reduce_min_sync(0xffffffffu, y0);
        x1 = __reduce_max_sync(0xffffffffu, x1);
        y1 = __reduce_max_sync(0xffffffffu, y1);
        flags = __reduce_or_sync(0xffffffffu, flags);
        if (lane == 0) {
            if (flags) {
                atomicOr(&scratch[0].z, flags);
                scratch[1 + p] = make_int4(0, 0, 0, 0);
            } else {
                int cx0 = max(x0, 0), cy0 = max(y0, 0), cx1 = min(x1, 65536), cy1 = min(y1, 65536);
                scratch[1 + p] = make_int4(cx0, cy0, max(cx1, cx0), max(cy1, cy0));
            }
        }
    }
}

__global__ void __launch_bounds__(kWarps * 32)
noalloc_sign_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off, uint64_t seed,
                    int K, uint32_t T, int chunks, int64_t n_items, int4* __restrict__ scratch,
                    uint32_t* __restrict__ out)
{
    __shared__ __align__(16) int2 sv[kWarps][kSmemVerts];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(&scratch[0]);
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(ticket, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= n_items) break;
        const int64_t p = (int64_t)(item / (unsigned)chunks);
        const int k0 = (int)(item % (unsigned)chunks) * 32;
        const int64_t b = off[p];
        const int n = (int)(off[p + 1] - b);
        const int4 bb = scratch[1 + p];
        const int2* v = xy + b;
        if (n <= kSmemVerts) {
            for (int i = lane; i < n; i += 32) sv[wid][i] = v[i];
            __syncwarp();
            v = sv[wid];
        }
        const uint32_t w = (uint32_t)(bb.z - bb.x), h = (uint32_t)(bb.w - bb.y);
        uint32_t mine = T;
        const int kend = min(K, k0 + 32);
        for (int k = k0; k < kend; ++k) {
            uint64_t sk = pmh_mix64(seed + (uint64_t)(k + 1) * PMH_GAMMA);
            uint32_t hk = sign_one(v, n, bb.x, bb.y, w, h, sk, T, lane);
            if (lane == k - k0) mine = hk;
        }
        if (k0 + lane < kend) out[p * (int64_t)K + k0 + lane] = mine;
        __syncwarp();
    }
}

struct NoallocDevice {
    int4* scratch = nullptr;  // device address of g_sign_scratch on this device
    int sm_count = 0;
    int blocks_per_sm = 0;
};
std::mutex g_noalloc_mutex;
NoallocDevice g_noalloc_dev[64];

}  // namespace

extern "C" int pmh_minhash_sign_noalloc(const int32_t* d_xy, const int64_t* d_offsets,
                                        int64_t n_polys, int64_t n_vertices,
                                        const pmh_params* params, uint32_t* d_hashes, void* stream)
{
    PMH_TRY(pmh_check_params(params));
    if (n_polys < 0 || n_vertices < 0 || !d_offsets || (n_polys > 0 && (!d_xy || !d_hashes)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (n_polys=%lld n_vertices=%lld)",
                             (long long)n_polys, (long long)n_vertices);
    if (n_polys > PMH_NOALLOC_MAX_POLYS)
        return pmh_set_error(PMH_ERR_RANGE,
                             "pmh_minhash_sign_noalloc handles at most %d polygons per call "
                             "(got %lld); split the batch or use pmh_minhash_sign",
                             PMH_NOALLOC_MAX_POLYS, (long long)n_polys);
    if (n_polys == 0) return PMH_OK;
    int dev = 0;
    PMH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return pmh_set_error(PMH_ERR_ARG, "device %d out of range", dev);
    // every array must be device (or managed) memory of the current device: a host
    // pointer, or memory of another GPU, is refused before anything is launched
    {
        const void* arrays[3] = {d_xy, d_offsets, d_hashes};
        const char* names[3] = {"d_xy", "d_offsets", "d_hashes"};
        for (int a = 0; a < 3; ++a) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, arrays[a]) != cudaSuccess) {
                cudaGetLastError();
                return pmh_set_error(PMH_ERR_ARG, "%s is not a CUDA pointer", names[a]);
            }
            const bool on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
            if (!on_device || (at.type == cudaMemoryTypeDevice && at.device != dev))
                return pmh_set_error(PMH_ERR_ARG,
                                     "%s must be device memory of the current device %d "
                                     "(memory type %d, device %d)",
                                     names[a], dev, (int)at.type, at.device);
        }
    }
    NoallocDevice nd;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocDevice& slot = g_noalloc_dev[dev];
        if (!slot.scratch) {  // once per device, with that device current
            void* p = nullptr;
            PMH_CUDA_TRY(cudaGetSymbolAddress(&p, g_sign_scratch));
            int sms = 0, per_sm = 0;
            PMH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_sign_kernel,
                                                                       kWarps * 32, 0));
            slot.sm_count = sms;
            slot.blocks_per_sm = per_sm > 0 ? per_sm : 1;
            slot.scratch = static_cast<int4*>(p);
        }
        nd = slot;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the ticket and the flags
    PMH_CUDA_TRY(cudaMemsetAsync(nd.scratch, 0, sizeof(int4), s));
    int prep_blocks = (int)std::min<int64_t>((n_polys + kWarps - 1) / kWarps, (int64_t)nd.sm_count * 16);
    noalloc_prep_kernel<<<prep_blocks, kWarps * 32, 0, s>>>(
        reinterpret_cast<const int2*>(d_xy), d_offsets, n_polys, n_vertices, nd.scratch);
    PMH_LAUNCHED("noalloc_prep_kernel");
    int4 head;
    PMH_CUDA_TRY(cudaMemcpyAsync(&head, nd.scratch, sizeof(int4), cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    if (head.z & 1) return pmh_set_error(PMH_ERR_RANGE, "offsets are not increasing / in range");
    if (head.z & 2) return pmh_set_error(PMH_ERR_RANGE, "a polygon has fewer than 3 vertices");
    if (head.z & 4) return pmh_set_error(PMH_ERR_RANGE, "a coordinate exceeds |2^20|");
    const int chunks = (int)((params->K + 31) / 32);
    const int64_t n_items = n_polys * chunks;
    int64_t blocks = (int64_t)nd.sm_count * nd.blocks_per_sm;
    blocks = std::min<int64_t>(blocks, (n_items + kWarps - 1) / kWarps);
    noalloc_sign_kernel<<<(int)blocks, kWarps * 32, 0, s>>>(
        reinterpret_cast<const int2*>(d_xy), d_offsets, params->seed, (int)params->K, params->T,
        chunks, n_items, nd.scratch, d_hashes);
    PMH_LAUNCHED("noalloc_sign_kernel");
    return PMH_OK;
}

// sign.cu -- step A1: MinHash signatures (Definition 2, Algorithm 1).
//
// h_k(P) = min{ i in [0,T) : point i of stream k lies in P }, else T.
//
// GB300 mapping.  The work is pure 32/64-bit integer arithmetic: the point
// generator (two 64-bit multiplies per point) dominates, the bbox test rejects
// almost every point, and the exact point-in-polygon test runs ~2-3 times per
// hash.  One warp owns a work item (polygon p, 32 consecutive hashes):
//   * the polygon's vertices are staged once into the warp's shared-memory
//     slice with 16-byte loads;
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
// SM count), which balances polygons whose expected work differs by 100x
// (Theorem 2: E[h] = 1/S_p).
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kWarps = 8;        // warps per block
constexpr int kSmemVerts = 256;  // vertices staged per warp (larger polygons read global)
constexpr int kU = 4;            // points per lane per round

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

// One hash of one polygon; every lane returns the same value.
__device__ __forceinline__ uint32_t sign_one(const int2* __restrict__ v, int n, int x0, int y0,
                                             uint32_t w, uint32_t h, uint64_t sk, uint32_t T,
                                             int lane)
{
    if (w == 0 || h == 0) return T;
    uint64_t z = sk + (uint64_t)(lane + 1) * PMH_GAMMA;
    const uint64_t step = 32ull * PMH_GAMMA;
    for (uint32_t i0 = 0; i0 < T; i0 += 32u * kU) {
        uint32_t pts[kU];
        unsigned m = 0;
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            uint32_t r = pmh_mix64_lo(z + (uint64_t)j * step);
            pts[j] = r;
            uint32_t dx = (r & 0xFFFFu) - (uint32_t)x0;
            uint32_t dy = (r >> 16) - (uint32_t)y0;
            m |= (unsigned)((dx < w) & (dy < h)) << j;
        }
        z += (uint64_t)kU * step;
        if (!__any_sync(0xffffffffu, m)) continue;
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            unsigned b = __ballot_sync(0xffffffffu, (m >> j) & 1u);
            while (b) {
                int l = __ffs(b) - 1;
                b &= b - 1;
                uint32_t i = i0 + (uint32_t)(j * 32 + l);
                if (i >= T) return T;
                uint32_t r = __shfl_sync(0xffffffffu, pts[j], l);
                if (warp_inside(v, n, (int)(r & 0xFFFFu), (int)(r >> 16), lane)) return i;
            }
        }
    }
    return T;
}

__global__ void __launch_bounds__(kWarps * 32)
sign_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
            const int4* __restrict__ bbox, uint64_t seed, int K, uint32_t T, int chunks,
            int64_t n_items, unsigned long long* __restrict__ ticket, uint32_t* __restrict__ out)
{
    __shared__ __align__(16) int2 sv[kWarps][kSmemVerts];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(ticket, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= n_items) break;
        const int64_t p = (int64_t)(item / (unsigned)chunks);
        const int k0 = (int)(item % (unsigned)chunks) * 32;
        const int64_t b = off[p];
        const int n = (int)(off[p + 1] - b);
        const int4 bb = bbox[p];
        const int2* v = xy + b;
        if (n <= kSmemVerts) {
            // stage vertices: 8-byte aligned source, so copy int2 by int2 (coalesced)
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

}  // namespace

extern "C" int pmh_minhash_sign(pmh_ctx ctx, pmh_polys polys, const pmh_params* params,
                                uint32_t* d_hashes, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (!polys || (!d_hashes && polys->n > 0))
        return pmh_set_error(PMH_ERR_ARG, "null polygons or output");
    if (polys->n == 0) return PMH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int chunks = (int)((params->K + 31) / 32);
    const int64_t n_items = polys->n * chunks;
    unsigned long long* ticket = ctx->d_tickets + 0;
    PMH_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    int per_sm = 0;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sign_kernel, kWarps * 32, 0));
    int64_t blocks = (int64_t)ctx->sm_count * std::max(per_sm, 1);
    blocks = std::min<int64_t>(blocks, (n_items + kWarps - 1) / kWarps);
    sign_kernel<<<(int)blocks, kWarps * 32, 0, s>>>(polys->xy, polys->offsets, polys->bbox,
                                                    params->seed, (int)params->K, params->T,
                                                    chunks, n_items, ticket, d_hashes);
    PMH_LAUNCHED("sign_kernel");
    return PMH_OK;
}

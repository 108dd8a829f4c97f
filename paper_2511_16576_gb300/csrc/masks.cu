// masks.cu -- per-polygon coverage masks (part of step A0, used by A1).
//
// A 16 x 16 grid of power-of-two cells covers the polygon's (clipped) bounding
// box: cell (i, j) holds the lattice points x0 + [i*cw, (i+1)*cw) by
// y0 + [j*ch, (j+1)*ch), with cw = 2^cwl the smallest power of two such that
// 16 * cw covers the box width (same for ch).  A cell whose closed rectangle,
// grown by one unit on its low sides, meets no edge of the polygon holds only
// lattice points of one membership (no edge separates them, and the e-shift of
// the half-open rule stays inside the grown rectangle); adjacent such cells in
// a row share that membership too.  So one exact membership test per run of
// untouched cells classifies them.  Codes (2 bits per cell, row j = word j):
//   0 every lattice point of the cell is outside, 1 every one is inside,
//   2 the boundary passes: use the exact test.
// Only polygons staged in shared memory by the signing kernel (<= 256
// vertices) get a mask; the others keep the exact test for every candidate.
#include <algorithm>

#include "sign_common.cuh"

namespace {

// exact half-open membership (same rule as the signing kernel), warp-cooperative
__device__ __forceinline__ bool warp_member(const int2* __restrict__ v, int n, int px, int py, int lane)
{
    unsigned par = 0;
    for (int e = lane; e < n; e += 32) {
        const int2 a = v[e], b = v[e + 1 == n ? 0 : e + 1];
        if ((a.y > py) != (b.y > py)) {
            const long long cr = (long long)(b.x - a.x) * (py - a.y) - (long long)(px - a.x) * (b.y - a.y);
            par ^= (cr != 0) & ((cr > 0) == (b.y > a.y));
        }
    }
    return __popc(__ballot_sync(0xffffffffu, par)) & 1;
}

constexpr int kMaskWarps = 8;

__global__ void __launch_bounds__(kMaskWarps * 32)
mask_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off, const int4* __restrict__ bbox,
            int64_t n_polys, int max_verts, uint32_t* __restrict__ masks)
{
    __shared__ int2 sv[kMaskWarps][kMaskMaxVerts];
    __shared__ uint32_t bnd[kMaskWarps][16];  // boundary bit per cell, row j = word j
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kMaskWarps;
    for (int64_t p = (int64_t)blockIdx.x * kMaskWarps + wid; p < n_polys; p += nwarps) {
        const int64_t b0 = off[p];
        const int n = (int)(off[p + 1] - b0);
        const int4 bb = bbox[p];
        uint32_t* out = masks + p * 16;
        if (n > max_verts || bb.z <= bb.x || bb.w <= bb.y) {
            if (lane < 16) out[lane] = 0xAAAAAAAAu;  // all cells "boundary": exact test
            continue;
        }
        for (int i = lane; i < n; i += 32) sv[wid][i] = xy[b0 + i];
        if (lane < 16) bnd[wid][lane] = 0;
        __syncwarp();
        const int cwl = mask_cell_log2(bb.z - bb.x), chl = mask_cell_log2(bb.w - bb.y);
        // 1) cells met by an edge
        for (int e = lane; e < n; e += 32) {
            const int2 a = sv[wid][e], c = sv[wid][e + 1 == n ? 0 : e + 1];
            // cells whose grown rectangle can meet the edge's box
            // (cell i's grown rectangle spans x - bb.x in [i*cw - 1, (i+1)*cw])
            const int ix0 = max(0, ((min(a.x, c.x) - bb.x) >> cwl) - 1);
            const int ix1 = min(15, (max(a.x, c.x) + 1 - bb.x) >> cwl);
            const int iy0 = max(0, ((min(a.y, c.y) - bb.y) >> chl) - 1);
            const int iy1 = min(15, (max(a.y, c.y) + 1 - bb.y) >> chl);
            for (int j = iy0; j <= iy1; ++j)
                for (int i = ix0; i <= ix1; ++i) {
                    const long long rx0 = (long long)bb.x + ((long long)i << cwl) - 1;
                    const long long rx1 = (long long)bb.x + ((long long)(i + 1) << cwl);
                    const long long ry0 = (long long)bb.y + ((long long)j << chl) - 1;
                    const long long ry1 = (long long)bb.y + ((long long)(j + 1) << chl);
                    if (seg_meets_rect(a, c, rx0, ry0, rx1, ry1)) atomicOr(&bnd[wid][j], 1u << i);
                }
        }
        __syncwarp();
        // 2) runs of untouched cells, one exact test each
        for (int j = 0; j < 16; ++j) {
            const uint32_t brow = bnd[wid][j];
            uint32_t word = 0;
            // cell codes: boundary cells 2
            for (int i = 0; i < 16; ++i)
                if ((brow >> i) & 1u) word |= 2u << (2 * i);
            uint32_t free_cells = ~brow & 0xFFFFu;
            while (free_cells) {
                const int s = __ffs(free_cells) - 1;
                int e = s;
                while (e + 1 < 16 && ((free_cells >> (e + 1)) & 1u)) ++e;
                const int px = bb.x + (s << cwl), py = bb.y + (j << chl);
                const bool in = warp_member(sv[wid], n, px, py, lane);
                if (in)
                    for (int i = s; i <= e; ++i) word |= 1u << (2 * i);
                free_cells &= ~(((2u << e) - 1u) & ~((1u << s) - 1u));
            }
            if (lane == 0) out[j] = word;
        }
        __syncwarp();
    }
}

}  // namespace

int pmh_build_masks(pmh_polys P, cudaStream_t s)
{
    if (P->n == 0) return PMH_OK;
    if (cudaMalloc(&P->mask, sizeof(uint32_t) * 16 * (size_t)P->n) != cudaSuccess) {
        cudaGetLastError();
        return pmh_set_error(PMH_ERR_NOMEM, "mask allocation failed");
    }
    const int blocks = (int)std::min<int64_t>((P->n + kMaskWarps - 1) / kMaskWarps,
                                              (int64_t)P->ctx->sm_count * 16);
    mask_kernel<<<blocks, kMaskWarps * 32, 0, s>>>(P->xy, P->offsets, P->bbox, P->n, kMaskMaxVerts,
                                                   P->mask);
    PMH_LAUNCHED("mask_kernel");
    return PMH_OK;
}

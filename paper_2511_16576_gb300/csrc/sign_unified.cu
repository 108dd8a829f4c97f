// sign_unified.cu -- step A1 (Definition 2, Algorithm 1): one persistent signing
// launch for polygons of every size, through the stream index.
//
// h_k(P) = min{ i : point i of stream k lies in P } is found, per polygon, in
// the indexed form or in the walk form, as the polygon's plan says
// (pmh_index_plan: the cheaper one by estimated warp instructions):
//   * indexed form: every point of stream k with index below the limit L that
//     falls in P's bounding box sits in one of the grid cells under the box
//     (stream_index.cu), and a cell record tells how many of its points lie
//     below each of six rank levels.  Sixteen hashes at a time, the (cell,
//     hash) records under the box are read one per lane, and the points they
//     hold are spread over the lanes by a warp scan (every lane loads one
//     point, no lane walks a list).  A point in the box is classified by the
//     polygon's 32 x 32 coverage mask: in an inside cell it is a hit and bounds
//     the hash from above, in an outside cell it is dropped, in a boundary
//     cell it is kept; kept points below their hash's smallest hit are tested
//     32 at a time, one per lane (lane-local exact test).  A hash without an
//     inside point below L (or whose kept points overflowed) walks on;
//   * walk form: Algorithm 1 in warp rounds of 32 * U consecutive stream
//     points; box candidates in index order (ballot + ffs), each decided by
//     the mask or by the warp-cooperative exact test.
// Edge sources: a polygon of at most 256 vertices is staged in the warp's
// shared-memory slice with its edges binned into 32 y-slabs; a larger one is
// read from global memory through the y-slab edge lists built at upload
// (slabs.cu), or through all its edges where it has none.  Either way an
// exact test reads only the edges of one slab.
//
// Work items come from one atomic ticket over a list of polygon slots: the
// first n_chunked slots are split into (polygon, 32-hash chunk) items -- the
// very large polygons (above 4,096 vertices), whose walks and tests cost the
// most, first and by decreasing cost -- and the remaining slots are whole
// polygons (all K hashes, so that the staging and the mask are paid once per
// polygon).  A
// staged polygon met in a chunked slot is signed whole by its chunk 0 (its
// other chunks return at once), so the captured query pipeline can hand in
// every polygon as a chunked slot.  Every step is exact, so the result equals
// the definition bit for bit.
#include <algorithm>
#include <type_traits>

#include "sign_common.cuh"

namespace {

// a kept point is packed as (hash within the group << 20 | stream index)
constexpr int kIdxBits = 20;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;
static_assert(kIndexMaxPoints <= (1 << kIdxBits), "point indices are packed in 20 bits");

constexpr int kUniWarps = 4;       // warps per block
constexpr int kUniMinBlocks = 8;   // resident blocks per SM the registers are sized for
constexpr int kSub = 16;           // hashes gathered together
constexpr int kMaskN = 32;         // coverage mask cells per side
constexpr int kPool = 256;         // kept (boundary) points of one group of kSub hashes
constexpr int kQueue = 64;         // exact-test queue (at most 31 + 32 entries)
constexpr int kIdxU = 4;           // points per lane per round of a resumed walk
constexpr int kMaskMaxEdges = 4096;  // larger polygons skip the mask (every cell is a boundary cell)

struct UniWarp {
    int2 v[kSmemVerts + 1];  // staged vertices, v[n] = v[0]
    uint8_t ids[kSlabCap];   // staged edges by slab
    uint16_t beg[kSlabs + 1];
    int cnt[kSlabs];
    uint32_t bnd[kMaskN];    // bit i of row j: an edge touches cell (i, j)
    uint32_t inb[kMaskN];    // bit i of row j: untouched cell (i, j) lies inside
    uint32_t best[kSub];     // per hash of the group: smallest inside index found
    uint2 pool[kPool];       // (hash << 20 | index, x | y << 16)
    uint2 queue[kQueue];
    int npool;
    uint32_t ovf;            // bit j: hash j lost kept points
};

// ---------------------------------------------------------------------------
// Edge sources.  vert(e) for e in [0, n] (vert(n) = vert(0)); row(py) gives the
// list positions [lo, hi) of the edges that can straddle the line y = py, and
// edge(t) the edge at list position t.
// ---------------------------------------------------------------------------
struct StagedSrc {
    const int2* v;
    const uint8_t* ids;
    const uint16_t* beg;
    int y0, sh;
    __device__ __forceinline__ int2 vert(int e) const { return v[e]; }
    __device__ __forceinline__ void row(int py, int& lo, int& hi) const
    {
        const int s = (py - y0) >> sh;
        lo = beg[s];
        hi = beg[s + 1];
    }
    __device__ __forceinline__ int edge(int t) const { return ids[t]; }
};

struct GlobalSrc {
    const int2* v;       // the polygon's first vertex
    int n;
    const int32_t* sp;   // slab table (nullptr: one list of every edge)
    const int32_t* se;   // edge lists
    int slab_h, ymin;
    __device__ __forceinline__ int2 vert(int e) const { return v[e == n ? 0 : e]; }
    __device__ __forceinline__ void row(int py, int& lo, int& hi) const
    {
        if (sp) {
            const int s = (py - ymin) / slab_h;
            lo = sp[s];
            hi = sp[s + 1];
        } else {
            lo = 0;
            hi = n;
        }
    }
    __device__ __forceinline__ int edge(int t) const { return sp ? se[t] : t; }
};

// exact half-open membership, one point per lane
template <class Src, class W>
__device__ __forceinline__ bool lane_inside(const Src& s, int px, int py, W& w)
{
    int lo, hi;
    s.row(py, lo, hi);
    w.lane_edges += hi - lo;
    unsigned par = 0;
    for (int t = lo; t < hi; ++t) {
        const int e = s.edge(t);
        par ^= edge_parity(s.vert(e), s.vert(e + 1), px, py);
    }
    return par;
}

// exact half-open membership, warp-cooperative (lanes split the row's edges)
template <class Src, class W>
__device__ __forceinline__ bool warp_inside_src(const Src& s, int px, int py, int lane, W& w)
{
    int lo, hi;
    s.row(py, lo, hi);
    w.edges += hi - lo;
    unsigned par = 0;
    for (int t = lo + lane; t < hi; t += 32) {
        const int e = s.edge(t);
        par ^= edge_parity(s.vert(e), s.vert(e + 1), px, py);
    }
    return __popc(__ballot_sync(0xffffffffu, par)) & 1;
}

__host__ __device__ __forceinline__ int mask32_log2(int w)
{
    int a = (w + kMaskN - 1) / kMaskN, l = 0;
    while ((1 << l) < a) ++l;
    return l;
}

// one slab holding every staged edge: the exact test then reads all n edges
__device__ __forceinline__ int single_slab(UniWarp& m, int n, int lane)
{
    for (int e = lane; e < n; e += 32) m.ids[e] = (uint8_t)e;
    if (lane == 0) m.beg[0] = 0;
    if (lane < kSlabs) m.beg[lane + 1] = (uint16_t)n;
    __syncwarp();
    return 16;
}

// 32 x 32 coverage mask over the clipped box bb (cell (i, j): lattice points
// bb.x + [i*cw, (i+1)*cw) by bb.y + [j*ch, (j+1)*ch)).  bnd marks every cell
// whose closed rectangle, grown by one unit on its low sides, meets an edge
// (and possibly a few neighbours: the marking is conservative).  Every lattice
// point of an unmarked cell (under the half-open reading, the point shifted up
// and right by an infinitesimal) then shares the membership of the whole
// rectangle.  Row j's unmarked cells are classified together from the edges
// crossing the line y = bb.y + j*ch: a cell is inside iff an odd number of
// crossings lies left of it.  A crossing lies in a marked cell of the row, at
// least one unit left of or strictly right of every unmarked cell, so its
// cell index -- computed in single precision, off by less than one unit --
// never moves it across an unmarked cell, and the classification is exact.
// Without a mask (use_mask false) every cell is a boundary cell.
template <class Src, class W>
__device__ __forceinline__ void build_mask(UniWarp& m, const Src& src, int n, int4 bb, int cwl,
                                           int chl, bool use_mask, int lane, W& work)
{
    if (!use_mask) {
        m.bnd[lane] = 0xFFFFFFFFu;
        m.inb[lane] = 0u;
        __syncwarp();
        return;
    }
    m.bnd[lane] = 0;
    __syncwarp();
    const float inv_cw = 1.0f / (float)(1 << cwl);
    const int ch = 1 << chl;
    for (int e = lane; e < n; e += 32) {
        const int2 a = src.vert(e), c = src.vert(e + 1);
        // rows whose grown band [j*ch - 1, (j+1)*ch] (relative) meets the edge's y-range
        const int ylo = min(a.y, c.y) - bb.y, yhi = max(a.y, c.y) - bb.y;
        const int j0 = max(0, ((ylo + ch - 1) >> chl) - 1);
        const int j1 = min(kMaskN - 1, (yhi + 1) >> chl);
        const float ax = (float)(a.x - bb.x), ay = (float)(a.y - bb.y);
        const float dx = (float)(c.x - a.x);
        const float inv_dy = c.y != a.y ? 1.0f / (float)(c.y - a.y) : 0.0f;
        for (int j = j0; j <= j1; ++j) {
            // the edge's x-range over the band (single precision, error < 1 unit)
            float t0 = 0.0f, t1 = 1.0f;
            if (c.y != a.y) {
                t0 = fminf(fmaxf(((float)((j << chl) - 1) - ay) * inv_dy, 0.0f), 1.0f);
                t1 = fminf(fmaxf(((float)((j + 1) << chl) - ay) * inv_dy, 0.0f), 1.0f);
            }
            const float xa = ax + dx * t0, xb = ax + dx * t1;
            // cells whose grown x-range [i*cw - 1, (i+1)*cw] meets it, one unit of margin
            const int i0 = max(0, (int)ceilf((fminf(xa, xb) - 1.0f) * inv_cw) - 1);
            const int i1 = min(kMaskN - 1, (int)floorf((fmaxf(xa, xb) + 2.0f) * inv_cw));
            if (i0 <= i1) {
                const uint32_t hi_bits = i1 == 31 ? 0xFFFFFFFFu : ((2u << i1) - 1u);
                atomicOr(&m.bnd[j], hi_bits & ~((1u << i0) - 1u));
            }
        }
    }
    __syncwarp();
    // lane j: parity of the crossings of the line y = bb.y + j*ch left of each cell
    // (rows below the box's top only: the slab lists cover [bb.y, bb.w))
    uint32_t word = 0;
    if ((lane << chl) < bb.w - bb.y) {
        const int py = bb.y + (lane << chl);
        int lo, hi;
        src.row(py, lo, hi);
        uint32_t par = 0;
        for (int t = lo; t < hi; ++t) {
            const int e = src.edge(t);
            const int2 a = src.vert(e), b = src.vert(e + 1);
            if ((a.y > py) != (b.y > py)) {
                const float x = (float)(a.x - bb.x) +
                                (float)(b.x - a.x) * ((float)(py - a.y) / (float)(b.y - a.y));
                const int ci = (int)floorf(x * inv_cw);
                par ^= ci < 0 ? 0xFFFFFFFFu : (ci >= kMaskN - 1 ? 0u : (0xFFFFFFFFu << (ci + 1)));
            }
        }
        work.lane_edges += hi - lo;
        word = par & ~m.bnd[lane];
    }
    m.inb[lane] = word;
    __syncwarp();
}

// Membership through the mask (warp-cooperative, for the walk form):
// untouched cells by their code, boundary cells by the exact test.
template <class Src>
struct MaskedWalker {
    const UniWarp* m;
    Src src;
    int x0, y0, cwl, chl;
    template <class W>
    __device__ __forceinline__ bool operator()(int px, int py, int lane, W& w) const
    {
        const int i = (px - x0) >> cwl, j = (py - y0) >> chl;
        if (!((m->bnd[j] >> i) & 1u)) {
            w.masked += 1;
            return (m->inb[j] >> i) & 1u;
        }
        return warp_inside_src(src, px, py, lane, w);
    }
};

// exact tests of queue[0 .. count), one per lane; an inside point lowers its hash's result
template <class Src, class W>
__device__ __forceinline__ void exact_batch(UniWarp& m, int count, const Src& src, int lane, W& work)
{
    if (lane < count) {
        const uint2 c = m.queue[lane];
        const int kl = (int)(c.x >> kIdxBits);
        const uint32_t idx = c.x & kIdxMask;
        if (idx < m.best[kl] && lane_inside(src, (int)(c.y & 0xFFFFu), (int)(c.y >> 16), work))
            atomicMin(&m.best[kl], idx);
    }
    __syncwarp();
}

// per-lane counts of the gather (widened at the end), and the same compiled away
struct GatherCounts {
    unsigned cells = 0, read = 0, cand = 0, masked = 0;
};
struct NoGather {
    Sink cells, read, cand, masked;
};

// Indexed form of hashes [k_begin, k_end) of polygon p (row `out` of the output).
template <class Src, class W, class G>
__device__ __forceinline__ void indexed_range(UniWarp& m, const Src& src, const StreamIndexView& S,
                                              PmhIndexPlan plan, int4 bb, uint64_t seed, uint32_t T,
                                              int k_begin, int k_end, uint32_t* __restrict__ out,
                                              int lane, W& work, G& gc)
{
    const unsigned full = 0xffffffffu;
    const uint32_t w = (uint32_t)(bb.z - bb.x), h = (uint32_t)(bb.w - bb.y);
    const int cwl = mask32_log2((int)w), chl = mask32_log2((int)h);
    uint32_t lim = min(plan.lim, T);
    // grid levels of the plan's two passes (coarser ones for boxes that span many
    // fine cells, the deep level for long walks); level 0 (second pass) or the
    // second pass's level (first pass) where that level is not built
    const int l2 = S.lv[plan.level].ranked && lim <= (uint32_t)S.lv[plan.level].M ? plan.level : 0;
    lim = min(lim, (uint32_t)S.lv[l2].M);  // every point below lim is in the level's lists
    const uint32_t lim1 = min(plan.lim1, lim);
    const int l1 = S.lv[plan.level1].ranked && lim1 <= (uint32_t)S.lv[plan.level1].M ? plan.level1 : l2;
    // first pass: the points below bound1 = M1 >> lev1, the smallest rank level >= lim1
    int lev1 = 0;
    while (lev1 + 1 < kRankLevels && ((uint32_t)S.lv[l1].M >> (lev1 + 1)) >= lim1) ++lev1;
    const uint32_t bound1 = (uint32_t)S.lv[l1].M >> lev1;
    // second pass: up to M2 >> lev (the smallest rank level >= lim), skipping the
    // points below bound1 when that is a rank level of its level (else reading
    // them again: they are outside the polygon or above their hash's bound)
    int lev = 0;
    while (lev + 1 < kRankLevels && ((uint32_t)S.lv[l2].M >> (lev + 1)) >= lim) ++lev;
    int lev_skip = -1;
    for (int t = lev; t < kRankLevels; ++t)
        if (((uint32_t)S.lv[l2].M >> t) == bound1) lev_skip = t;
    const bool second = ((uint32_t)S.lv[l2].M >> lev) > bound1;
    const MaskedWalker<Src> walker{&m, src, bb.x, bb.y, cwl, chl};
    const int hl = lane & (kSub - 1);

    for (int kc = k_begin; kc < k_end; kc += kSub) {
        const int kn = min(kSub, k_end - kc);
        if (lane < kSub) m.best[lane] = 0xFFFFFFFFu;
        if (lane == 0) m.ovf = 0;
        // two passes over the cells: first the points below level lev1 (about
        // 3.5x the expected first hit: most hashes find their answer there),
        // then, for the hashes with no inside point yet, those up to level lev
        uint32_t open = kn == 32 ? 0xFFFFFFFFu : ((1u << kn) - 1u);
        for (int pass = 0; pass < 2 && lim > 0; ++pass) {
            const int hi_lev = pass == 0 ? lev1 : lev;       // read entries below M >> hi_lev
            const int lo_lev = pass == 0 ? -1 : lev_skip;    // ... skipping those below M >> lo_lev
            if (pass == 1 && (!second || open == 0)) break;
            // the pass's grid level: cells under the box, row-major; a round reads two
            // cells for the kSub hashes of a group (lane: hash lane & 15, cell
            // 2 * round + lane / 16)
            const IndexLevelView& L = S.lv[pass == 0 ? l1 : l2];
            const uint2* cells = L.cell;
            const uint2* ents = L.ent;
            const int gb = L.gbits, shf = L.shift;
            const int cx0 = bb.x >> shf, cy0 = bb.y >> shf;
            const int ncx = ((bb.z - 1) >> shf) - cx0 + 1;
            const int C = ncx * (((bb.w - 1) >> shf) - cy0 + 1);
            if (lane == 0) m.npool = 0;
            __syncwarp();
            const bool mine = hl < kn && ((open >> hl) & 1u);
            const uint2* rec = cells + kc + hl;
            int cx = lane >> 4, cy = 0;
            if (cx >= ncx) {
                cx -= ncx;
                ++cy;
            }
            if (lane == 0) gc.cells += (unsigned)(C * __popc(open));
            // the records of the next round are loaded while this round's points are read
            uint2 rnext = make_uint2(0u, 0u);
            if ((lane >> 4) < C && mine) rnext = rec[(int64_t)(((cy0 + cy) << gb) | (cx0 + cx)) * S.K];
            for (int c0 = 0; c0 < C; c0 += 2) {
                // one (hash, cell) record per lane: its points between the levels
                const uint2 r = rnext;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    cx += 1;
                    if (cx >= ncx) {
                        cx -= ncx;
                        ++cy;
                    }
                }
                rnext = make_uint2(0u, 0u);
                if (c0 + 2 + (lane >> 4) < C && mine)
                    rnext = rec[(int64_t)(((cy0 + cy) << gb) | (cx0 + cx)) * S.K];
                const uint32_t below_lo = lo_lev < 0 ? 0u : (r.y >> (5 * lo_lev)) & 31u;
                const uint32_t first = r.x + below_lo, cnt = ((r.y >> (5 * hi_lev)) & 31u) - below_lo;
                uint32_t incl = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(full, incl, d);
                    if (lane >= d) incl += t;
                }
                const uint32_t excl = incl - cnt;
                const int E = (int)__shfl_sync(full, incl, 31);
                gc.read += lane == 0 ? (unsigned)E : 0u;
                // spread the points over the lanes: point e belongs to the last
                // lane whose exclusive offset is <= e
                for (int e0 = 0; e0 < E; e0 += 32) {
                    const uint32_t e = (uint32_t)(e0 + lane);
                    int own = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1)
                        if (__shfl_sync(full, excl, own + step) <= e) own += step;
                    const uint32_t o_first = __shfl_sync(full, first, own);
                    const uint32_t o_excl = __shfl_sync(full, excl, own);
                    const int o_hl = own & (kSub - 1);
                    if ((int)e < E) {
                        const uint2 q = ents[o_first + (e - o_excl)];
                        const uint32_t rr = q.y;
                        const uint32_t dx = (rr & 0xFFFFu) - (uint32_t)bb.x;
                        const uint32_t dy = (rr >> 16) - (uint32_t)bb.y;
                        if (q.x < lim && dx < w && dy < h) {
                            ++gc.cand;
                            const int i = (int)(dx >> cwl), j = (int)(dy >> chl);
                            if ((m.bnd[j] >> i) & 1u) {
                                const int slot = atomicAdd(&m.npool, 1);
                                if (slot < kPool) m.pool[slot] = make_uint2(((uint32_t)o_hl << kIdxBits) | q.x, rr);
                                else atomicOr(&m.ovf, 1u << o_hl);
                            } else {
                                ++gc.masked;
                                if ((m.inb[j] >> i) & 1u) atomicMin(&m.best[o_hl], q.x);
                            }
                        }
                    }
                }
            }
            __syncwarp();
            // kept points below their hash's smallest hit go to the queue, tested 32 at a time
            const int np = min(m.npool, kPool);
            int nq = 0;  // warp-uniform queue length
            for (int t0 = 0; t0 < np; t0 += 32) {
                const int t = t0 + lane;
                uint2 c = make_uint2(0u, 0u);
                bool keep = false;
                if (t < np) {
                    c = m.pool[t];
                    keep = (c.x & kIdxMask) < m.best[c.x >> kIdxBits];
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) m.queue[nq + __popc(bal & pmh_lanemask_lt())] = c;
                nq += __popc(bal);
                __syncwarp();
                if (nq >= 32) {
                    exact_batch(m, 32, src, lane, work);
                    nq -= 32;
                    const uint2 rest = lane < nq ? m.queue[32 + lane] : make_uint2(0u, 0u);
                    __syncwarp();
                    if (lane < nq) m.queue[lane] = rest;
                    __syncwarp();
                }
            }
            if (nq > 0) exact_batch(m, nq, src, lane, work);
            // a hash with an inside point below the first level is final (every point
            // below it was examined); one that lost kept points walks from the start
            open &= __ballot_sync(full, lane < kn && m.best[lane] == 0xFFFFFFFFu) & ~m.ovf;
        }

        // hashes without an inside point below lim resume the walk there; one
        // that lost kept points walks from the start
        const uint32_t overs = m.ovf;
        unsigned todo =
            __ballot_sync(full, lane < kn && (((overs >> lane) & 1u) || m.best[lane] == 0xFFFFFFFFu));
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t start = ((overs >> j) & 1u) ? 0u : lim;
            uint32_t hk = T;
            if (start < T) {
                const uint64_t sk = pmh_mix64(seed + (uint64_t)(kc + j + 1) * PMH_GAMMA);
                hk = sign_one_t<kIdxU>(walker, bb.x, bb.y, w, h, sk, T, lane, work, start);
            }
            if (lane == 0) m.best[j] = hk;
        }
        __syncwarp();
        if (lane < kn) out[kc + lane] = m.best[lane];
        __syncwarp();
    }
}

// Walk form of hashes [k_begin, k_end): lane j keeps hash k0 + j of each 32.
template <int U, class Src, class W>
__device__ __forceinline__ void walk_range(const UniWarp& m, const Src& src, int4 bb, uint64_t seed,
                                           uint32_t T, int k_begin, int k_end,
                                           uint32_t* __restrict__ out, int lane, W& work)
{
    const uint32_t w = (uint32_t)(bb.z - bb.x), h = (uint32_t)(bb.w - bb.y);
    const MaskedWalker<Src> walker{&m, src, bb.x, bb.y, mask32_log2((int)w), mask32_log2((int)h)};
    for (int k0 = k_begin; k0 < k_end; k0 += 32) {
        const int kend = min(k_end, k0 + 32);
        uint32_t mine = T;
        for (int k = k0; k < kend; ++k) {
            const uint64_t sk = pmh_mix64(seed + (uint64_t)(k + 1) * PMH_GAMMA);
            const uint32_t hk = sign_one_t<U>(walker, bb.x, bb.y, w, h, sk, T, lane, work);
            if (lane == k - k0) mine = hk;
        }
        if (k0 + lane < kend) out[k0 + lane] = mine;
    }
}

// Walk form of a staged polygon, kept out of line so that its registers do not
// weigh on the indexed form's gather (Work by pointer: a local copy inside).
template <int U, class W>
__device__ __noinline__ void walk_staged(const UniWarp& m, StagedSrc src, int4 bb, uint64_t seed,
                                         uint32_t T, int k_begin, int k_end, uint32_t* out,
                                         int lane, W* work)
{
    W local;
    walk_range<U>(m, src, bb, seed, T, k_begin, k_end, out, lane, local);
    work->walk += local.walk;
    work->cand += local.cand;
    work->edges += local.edges;
    work->masked += local.masked;
    work->lane_edges += local.lane_edges;
}

// A polygon above the staged size (read from global memory): the mask, then the
// planned form, out of line for the same reason.
template <int U, class W, class G>
__device__ __noinline__ void sign_global(UniWarp& m, GlobalSrc src, int n, int4 bb, PmhIndexPlan plan,
                                         const StreamIndexView& S, uint64_t seed, uint32_t T,
                                         int k_begin, int k_end, uint32_t* out, int lane, W* work,
                                         G* gc)
{
    W local;
    G g;
    build_mask(m, src, n, bb, mask32_log2(bb.z - bb.x), mask32_log2(bb.w - bb.y), n <= kMaskMaxEdges,
               lane, local);
    if (plan.lim > 0)
        indexed_range(m, src, S, plan, bb, seed, T, k_begin, k_end, out, lane, local, g);
    else
        walk_range<U>(m, src, bb, seed, T, k_begin, k_end, out, lane, local);
    work->walk += local.walk;
    work->cand += local.cand;
    work->edges += local.edges;
    work->masked += local.masked;
    work->lane_edges += local.lane_edges;
    gc->cells += g.cells;
    gc->read += g.read;
    gc->cand += g.cand;
    gc->masked += g.masked;
}

// kIndexedOnly: a launch over staged polygons of the indexed form only (the class
// order's last class), compiled without the walk-form and large-polygon paths, so that
// the gather keeps its values in registers (a fraction of the unified build's spills
// and no call frames)
template <int U, bool kCount, bool kIndexedOnly>
__global__ void __launch_bounds__(kUniWarps * 32, kUniMinBlocks)
sign_unified_kernel(const int2* __restrict__ xy, const int64_t* __restrict__ off,
                    const int4* __restrict__ bbox, const int64_t* __restrict__ area2,
                    const SlabInfo* __restrict__ slabs, const int32_t* __restrict__ slab_ptr,
                    const int32_t* __restrict__ slab_edges, const int32_t* __restrict__ list,
                    int64_t n_slots, int64_t n_chunked, const int64_t* __restrict__ d_n,
                    const int* __restrict__ d_flags, uint64_t seed, int K, uint32_t T,
                    StreamIndexView S, unsigned long long* __restrict__ ticket,
                    uint32_t* __restrict__ out, unsigned long long* __restrict__ work_out)
{
    __shared__ UniWarp smem[kUniWarps];
    __shared__ unsigned long long wsum[6];
    if (threadIdx.x < 6) wsum[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    UniWarp& m = smem[threadIdx.x >> 5];
    const unsigned full = 0xffffffffu;
    // work counters only in launches that report them
    using W = typename std::conditional<kCount, Work, NoWork>::type;
    using G = typename std::conditional<kCount, GatherCounts, NoGather>::type;
    W work;
    G gc;
    const bool failed = d_flags && *d_flags;  // the batch failed validation
    if (d_n) n_slots = min(n_slots, *d_n);
    n_chunked = min(n_chunked, n_slots);
    const int chunks = (K + 31) / 32;
    const int64_t n_items = failed ? 0 : n_chunked * chunks + (n_slots - n_chunked);
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(ticket, 1ull);
        item = __shfl_sync(full, item, 0);
        if ((int64_t)item >= n_items) break;
        int64_t slot;
        int chunk = -1;  // -1: the whole polygon
        if ((int64_t)item < n_chunked * chunks) {
            slot = (int64_t)item / chunks;
            chunk = (int)((int64_t)item - slot * chunks);
        } else {
            slot = n_chunked + ((int64_t)item - n_chunked * chunks);
        }
        const int64_t p = list ? (int64_t)list[slot] : slot;
        const int64_t b = off[p];
        const int n = (int)(off[p + 1] - b);
        const bool staged = n <= kSmemVerts;
        if (staged && chunk > 0) continue;  // signed whole by its chunk 0
        const int k_begin = (staged || chunk < 0) ? 0 : 32 * chunk;
        const int k_end = (staged || chunk < 0) ? K : min(K, 32 * chunk + 32);
        uint32_t* row = out + p * (int64_t)K;
        const int4 bb = bbox[p];
        if (bb.z <= bb.x || bb.w <= bb.y) {  // no lattice point in the box: every hash is T
            for (int k = k_begin + lane; k < k_end; k += 32) row[k] = T;
            continue;
        }
        // the form (indexed or walk) and grid level the polygon's cost model picks
        const PmhIndexPlan plan = (S.cell && area2) ? pmh_index_plan(bb, area2[p]) : PmhIndexPlan{0u, 0, 0u, 0};
        if (staged) {
            // stage the polygon (closed: v[n] = v[0]; cp.async 8-byte copies) and bin its edges
            stage_vertices(m.v, xy + b, n, lane);
            int sh = staged_slab_shift(bb.w - bb.y);
            if (!build_staged_slabs(m.v, n, bb.y, sh, m.ids, m.beg, m.cnt, lane)) sh = single_slab(m, n, lane);
            const StagedSrc src{m.v, m.ids, m.beg, bb.y, sh};
            build_mask(m, src, n, bb, mask32_log2(bb.z - bb.x), mask32_log2(bb.w - bb.y), true, lane,
                       work);
            if (kIndexedOnly || plan.lim > 0)
                indexed_range(m, src, S, plan, bb, seed, T, k_begin, k_end, row, lane, work, gc);
            else
                walk_staged<U, W>(m, src, bb, seed, T, k_begin, k_end, row, lane, &work);
        } else if (!kIndexedOnly) {
            const SlabInfo si = slabs ? slabs[p] : SlabInfo{0, 0, 0, 1, 0};
            const GlobalSrc src{xy + b, n, si.S > 0 ? slab_ptr + si.slab_base : nullptr,
                                si.S > 0 ? slab_edges + si.edge_base : nullptr, si.slab_h, si.ymin};
            sign_global<U, W, G>(m, src, n, bb, plan, S, seed, T, k_begin, k_end, row, lane, &work, &gc);
        }
        __syncwarp();
    }
    if (kCount && work_out) {
        unsigned long long le = work.lane_edges, en = gc.read, ca = gc.cand, ma = gc.masked,
                           ce = gc.cells;  // (the gather's 32-bit lane counts, widened)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            le += __shfl_xor_sync(full, le, o);
            en += __shfl_xor_sync(full, en, o);
            ca += __shfl_xor_sync(full, ca, o);
            ma += __shfl_xor_sync(full, ma, o);
            ce += __shfl_xor_sync(full, ce, o);
        }
        if (lane == 0) {
            // Work's walk, candidates, edges and masked counts are warp-uniform; the
            // gather's counts and the lane-local edge tests are per lane
            atomicAdd(&wsum[0], work.walk);
            atomicAdd(&wsum[1], ce);
            atomicAdd(&wsum[2], en);
            atomicAdd(&wsum[3], ca + work.cand);
            atomicAdd(&wsum[4], work.edges + le);
            atomicAdd(&wsum[5], ma + work.masked);
        }
        __syncthreads();
        if (threadIdx.x < 6) atomicAdd(&work_out[threadIdx.x], wsum[threadIdx.x]);
    }
}

}  // namespace

// one persistent launch over `n` slots of `list` (or slot order) with its own ticket
template <bool kIndexedOnly>
static int launch_unified(pmh_ctx ctx, int U, const int2* xy, const int64_t* off, const int4* bbox,
                          const int64_t* area2, const SlabInfo* slabs, const int32_t* slab_ptr,
                          const int32_t* slab_edges, const int32_t* list, int64_t n_slots,
                          int64_t n_chunked, const int64_t* d_n, const int* d_flags, const pmh_params* P,
                          const StreamIndexView& S, unsigned long long* ticket, uint32_t* out,
                          unsigned long long* work, cudaStream_t s)
{
    auto fn = kIndexedOnly
                  ? (work ? sign_unified_kernel<2, true, true> : sign_unified_kernel<2, false, true>)
                  : work ? (U <= 2   ? sign_unified_kernel<2, true, false>
                            : U <= 4 ? sign_unified_kernel<4, true, false>
                                     : sign_unified_kernel<8, true, false>)
                         : (U <= 2   ? sign_unified_kernel<2, false, false>
                            : U <= 4 ? sign_unified_kernel<4, false, false>
                                     : sign_unified_kernel<8, false, false>);
    int per_sm = 0;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kUniWarps * 32, 0));
    const int chunks = (int)((P->K + 31) / 32);
    const int64_t n_items = n_chunked * chunks + (n_slots - n_chunked);
    int64_t blocks = (int64_t)ctx->sm_count * std::max(per_sm, 1);
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (n_items + kUniWarps - 1) / kUniWarps));
    PMH_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    fn<<<(int)blocks, kUniWarps * 32, 0, s>>>(xy, off, bbox, area2, slabs, slab_ptr, slab_edges, list,
                                              n_slots, n_chunked, d_n, d_flags, P->seed, (int)P->K,
                                              P->T, S, ticket, out, work);
    PMH_LAUNCHED(kIndexedOnly ? "sign_unified_kernel<indexed>" : "sign_unified_kernel");
    return PMH_OK;
}

int pmh_launch_sign_unified(pmh_ctx ctx, int U, const int2* xy, const int64_t* off,
                            const int4* bbox, const int64_t* area2, const SlabInfo* slabs,
                            const int32_t* slab_ptr, const int32_t* slab_edges, const int32_t* list,
                            int64_t n_slots, int64_t n_chunked, int64_t n_indexed_tail,
                            const int64_t* d_n, const int* d_flags, const pmh_params* P,
                            const StreamIndexView& S, unsigned long long* ticket, uint32_t* out,
                            unsigned long long* work, cudaStream_t s)
{
    if (n_slots <= 0) return PMH_OK;
    // the indexed class at the list's end goes to its own launch (needs the class list)
    const int64_t tail = list && !d_n ? std::min(std::max<int64_t>(n_indexed_tail, 0), n_slots - n_chunked) : 0;
    if (n_slots - tail > 0)
        PMH_TRY(launch_unified<false>(ctx, U, xy, off, bbox, area2, slabs, slab_ptr, slab_edges, list,
                                      n_slots - tail, n_chunked, d_n, d_flags, P, S, ticket, out, work, s));
    if (tail > 0)
        PMH_TRY(launch_unified<true>(ctx, U, xy, off, bbox, area2, slabs, slab_ptr, slab_edges,
                                     list + (n_slots - tail), tail, 0, nullptr, d_flags, P, S, ticket, out,
                                     work, s));
    return PMH_OK;
}

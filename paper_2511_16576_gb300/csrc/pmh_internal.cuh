// pmh_internal.cuh -- internal declarations of the PolyMinHash CUDA library.
//
// Shared by the library's translation units only (never by the CPU oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/polyminhash.h"

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
int pmh_set_error(int code, const char* fmt, ...);
#define PMH_CUDA_TRY(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return pmh_set_error(PMH_ERR_CUDA, "%s failed: %s (%s:%d)", #call,         \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);          \
    } while (0)
#define PMH_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != PMH_OK) return rc_; \
    } while (0)

extern std::atomic<int64_t> g_pmh_launches;
// launch bookkeeping: count every kernel launch and check the launch status
#define PMH_LAUNCHED(name)                                                              \
    do {                                                                                \
        g_pmh_launches.fetch_add(1, std::memory_order_relaxed);                         \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return pmh_set_error(PMH_ERR_CUDA, "launch of %s failed: %s", name,         \
                                 cudaGetErrorString(e_));                               \
    } while (0)

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
enum ScratchSlot {
    SCR_SORT_A = 0,
    SCR_SORT_B,
    SCR_SORT_HIST,
    SCR_SCAN,
    SCR_QUERY,
    SCR_REFINE,
    SCR_MISC,
    SCR_JOIN,
    SCR_COUNT
};

// first kStreamIndexPoints points of every hash's stream, bucketed by cell of a
// 2^kStreamGridBits-square grid (stream_index.cu); the other levels hold fewer
// points on coarser grids or more points on a finer one (level l:
// 2^index_level_gbits(l) cells per side, the first index_level_points(l)
// points): 65,536 on 128^2, 32,768 on 64^2, 8,192 on 32^2 and 2^20 on 512^2
// (about four points per (cell, hash) list on levels 0 and 3, eight on 1 and 2)
constexpr int kStreamGridBits = 7;
constexpr int kStreamIndexPoints = 65536;
constexpr int kIndexLevels = 4;
constexpr int kIndexMaxPoints = 1 << 20;  // the deepest level
__host__ __device__ constexpr int index_level_gbits(int l) { return l == 0 ? 7 : l == 1 ? 6 : l == 2 ? 5 : 9; }
__host__ __device__ constexpr int index_level_points(int l)
{
    return l == 0 ? 65536 : l == 1 ? 32768 : l == 2 ? 8192 : kIndexMaxPoints;
}
// a level is built only if its entry offsets (K * points) fit in 31 bits
__host__ __device__ constexpr bool index_level_fits(int l, int K)
{
    return (long long)K * index_level_points(l) <= (1ll << 31);
}
// polygons of at most this many vertices are staged in shared memory by the
// signing kernels; larger ones are read through their y-slab edge index
constexpr int kStagedMaxVerts = 256;
// polygons above this many vertices are signed in (polygon, 32-hash chunk) items, so that
// a few very large polygons spread over many warps; smaller ones are signed whole (the
// staging, slab lists and coverage mask are then built once per polygon)
constexpr int kChunkMinVerts = 4096;

// Cost model of the indexed form for one polygon (clipped box bb, twice its
// area), in warp instructions per hash: the walk examines about 2^32 / area
// points, 128 per round of ~130 instructions; the indexed form reads the cells
// under the bounding box, 32 per round of ~50 instructions, and sees about
// lim * bbox / 2^32 candidates, with lim = 8 * 2^32 / area (a hit is then
// missed with probability ~e^-8 and the walk resumes at lim).  Returns lim, or
// 0 to walk.  The same function decides the class of a polygon at upload and
// the limit in the signing kernels.
__host__ __device__ __forceinline__ uint32_t pmh_indexed_limit(int4 bb, long long area2)
{
    // single precision: the estimate only picks a form and a limit (any limit
    // gives the exact result), and double precision is slow on this GPU
    if (bb.z <= bb.x || bb.w <= bb.y) return 0;
    const int shift = 16 - kStreamGridBits;
    const float area = 0.5f * (float)(area2 < 0 ? -area2 : area2);
    const float walk = 4294967296.0f / fmaxf(area, 1.0f);
    const float cells = (float)((((bb.z - 1) >> shift) - (bb.x >> shift) + 1) *
                                (((bb.w - 1) >> shift) - (bb.y >> shift) + 1));
    const float lim = fminf((float)kStreamIndexPoints, 8.0f * walk + 256.0f);
    const float cand = lim * ((float)(bb.z - bb.x) * (float)(bb.w - bb.y) * (1.0f / 4294967296.0f));
    const float walk_cost = ceilf(walk * (1.0f / 128.0f)) * 130.0f;
    const float index_cost = ceilf(cells * (1.0f / 32.0f)) * 50.0f + 40.0f;
    if (index_cost >= walk_cost || cand > 24.0f) return 0;
    return (uint32_t)lim;
}

// Cell records of the stream index, cell-major: record (cell c, hash k) is
// cell[c * K + k]; .x = first entry of the list of (k, c), which ends where
// record (c + 1, k) starts (row c = G*G is the end of every hash's lists);
// .y = six 5-bit counts, bits [5t, 5t+5) = entries of the list with stream
// index below M >> t.  The records of one cell for consecutive hashes are
// adjacent, so a warp reading one cell for sixteen hashes reads 128 bytes.
constexpr int kRankLevels = 6;
// Plan of the indexed form for a polygon (sign_unified.cu),
// in estimated warp instructions per hash.  The limit is lim = 11 * 2^32 / area (a
// hit below it is missed with probability ~e^-11; the walk then resumes at lim),
// capped at the shallow levels' 65,536 points where 8 * 2^32 / area fits there, and
// at most ~24 box points below 8 * 2^32 / area are expected.  The gather first reads the
// points below lim1 = 3.5 * 2^32 / area (an inside point exists there with
// probability ~1 - e^-3.5); only the hashes without one read on up to lim.  On a
// grid level holding at least lim points it costs ~4.9 per cell record under the
// box and ~2.5 per first-pass point read (those below the smallest rank level >=
// lim1 in those cells), plus ~20 for the mask, exact tests and setup; the walk
// costs ~45 per round of 64 points plus ~40.  Returns lim (0 = walk), lim1 and
// the cheapest level for each pass.  Any limit and levels give the exact result;
// the plan only picks the cheaper work.
struct PmhIndexPlan {
    uint32_t lim;
    int level;      // grid level holding every point below lim (the second pass)
    uint32_t lim1;  // bound of the first gather pass: ~3.5 expected first hits
    int level1;     // grid level of the first pass (holding every point below lim1)
};
__host__ __device__ __forceinline__ float pmh_level_cost(int4 bb, uint32_t lim1, uint32_t M, int shift)
{
    const float C = (float)((((bb.z - 1) >> shift) - (bb.x >> shift) + 1) *
                            (((bb.w - 1) >> shift) - (bb.y >> shift) + 1));
    uint32_t lvl = M;
    for (int t = 1; t < 6 && (M >> t) >= lim1; ++t) lvl = M >> t;
    const float pts = (float)lvl * C * (float)(1u << (2 * shift)) * (1.0f / 4294967296.0f);
    return 4.9f * C + 2.5f * pts;
}
__host__ __device__ __forceinline__ PmhIndexPlan pmh_index_plan(int4 bb, long long area2)
{
    PmhIndexPlan plan{0u, 0, 0u, 0};
    if (bb.z <= bb.x || bb.w <= bb.y) return plan;
    const float area = 0.5f * (float)(area2 < 0 ? -area2 : area2);
    const float walk = 4294967296.0f / fmaxf(area, 1.0f);
    // a polygon is indexed when ~24 box points lie below 8 expected first hits; its limit
    // is 11 of them, but not past the shallow levels' 65,536 points when 8 fit there
    const float lim8 = 8.0f * walk + 256.0f;
    float lim = fminf((float)kIndexMaxPoints, 11.0f * walk + 256.0f);
    if (lim8 <= (float)kStreamIndexPoints) lim = fminf(lim, (float)kStreamIndexPoints);
    const float box = (float)(bb.z - bb.x) * (float)(bb.w - bb.y) * (1.0f / 4294967296.0f);
    if (fminf((float)kIndexMaxPoints, lim8) * box > 24.0f) return plan;
    const uint32_t L = (uint32_t)lim, L1 = (uint32_t)fminf(lim, 3.5f * walk + 64.0f);
    // the cheapest level holding every point below the bound: L for the second pass,
    // L1 for the first (on a coarser shallow level the first pass reads a few cells
    // where the deep level holding L would read many); the deep level (larger than
    // L2) only for bounds the L2-resident levels cannot hold
    float best = 3.0e38f, best1 = 3.0e38f;
    int level = 0, level1 = 0;
    for (int l = 0; l < kIndexLevels; ++l) {
        const uint32_t M = (uint32_t)index_level_points(l);
        const bool deep = M > (uint32_t)kStreamIndexPoints;
        const float c = pmh_level_cost(bb, L1, M, 16 - index_level_gbits(l));
        if (L <= M && !(deep && L <= (uint32_t)kStreamIndexPoints) && c < best) {
            best = c;
            level = l;
        }
        if (L1 <= M && !(deep && L1 <= (uint32_t)kStreamIndexPoints) && c < best1) {
            best1 = c;
            level1 = l;
        }
    }
    const float walk_cost = ceilf(walk * (1.0f / 64.0f)) * 45.0f + 40.0f;
    if (best1 + 20.0f >= walk_cost) return plan;
    plan.lim = L;
    plan.level = level;
    plan.lim1 = L1;
    plan.level1 = level1;
    return plan;
}

struct StreamIndex {
    uint64_t seed = 0;
    int K = 0;
    uint2* cell[kIndexLevels] = {};  // per level: [(G * G + 1) * K] records
    uint2* ent[kIndexLevels] = {};   // per level: [K * M] (stream index, x | y << 16)
    int ranked[kIndexLevels] = {};   // every list of the level fits the 5-bit counts
};
struct IndexLevelView {
    const uint2* cell;
    const uint2* ent;
    int M, gbits, shift, ranked;
};
struct StreamIndexView {
    const uint2* cell;  // level 0 (nullptr: no index)
    const uint2* ent;
    int M, gbits, shift, ranked, K;
    IndexLevelView lv[kIndexLevels];
};

struct pmh_ctx_s {
    int device = 0;
    int sm_count = 0;
    int* d_status = nullptr;              // device status word (0 = ok)
    unsigned long long* d_tickets = nullptr;  // work-queue tickets [64]
    void* scratch[SCR_COUNT] = {};
    size_t scratch_bytes[SCR_COUNT] = {};
    int64_t* h_pinned = nullptr;          // small pinned host buffer [64]
    int sign_variant = -1;                // autotuned signing kernel (-1 = default)
    StreamIndex sindex;                   // cached stream index (PMH_FLAG_STREAM_INDEX)
    int sign_timing = 0;                  // record per-kernel events in pmh_minhash_sign
    int sign_count = 1;                   // signing launches record their work counts
    std::vector<cudaEvent_t> sign_ev;     // three per recorded call
    size_t sign_ev_used = 0;
};

int pmh_stream_index_get(pmh_ctx ctx, const pmh_params* P, cudaStream_t s, StreamIndexView* out);

// per-polygon y-slab edge index (slabs.cu); S == 0 for polygons without one
struct SlabInfo {
    int64_t slab_base;  // first entry of the polygon's slab table in slab_ptr
    int64_t edge_base;  // first entry of its edge lists in slab_edges
    int32_t S;          // number of slabs
    int32_t slab_h;     // slab height (rows)
    int32_t ymin;       // lowest vertex y
};
constexpr int kSlabMinVerts = 256;  // polygons above this size get a slab index

// Handles record their device so that they can be released after their context.
struct pmh_polys_s {
    pmh_ctx ctx = nullptr;
    int device = 0;
    int64_t n = 0, nv = 0;
    int2* xy = nullptr;
    int64_t* offsets = nullptr;
    int4* bbox = nullptr;      // x0, y0, x1, y1 half-open, clipped to the domain
    int64_t* area2 = nullptr;  // twice the signed area
    int32_t max_n = 0;         // largest vertex count
    float2* feat = nullptr;         // [n] log2(area) / 32, log2(n) / 16 (reranker inputs)
    SlabInfo* slab_info = nullptr;  // [n]
    int32_t* slab_ptr = nullptr;
    int32_t* slab_edges = nullptr;
    int32_t* order = nullptr;       // polygons by expected signing cost, largest first (built
                                    // on the first signing call without the stream index)
    int32_t* order_cls = nullptr;   // class order: polygons above kChunkMinVerts vertices, then
                                    // the other polygons signed in cost order (staged walk-form
                                    // ones and those above kStagedMaxVerts), each by cost, then
                                    // staged indexed-form polygons (Morton order)
    int64_t n_indexed = 0;          // class 0: <= kStagedMaxVerts vertices, pmh_index_plan lim > 0
    int64_t n_whole_cost = 0;       // class 1: the rest up to kChunkMinVerts vertices
    uint32_t* mask = nullptr;       // [n][16] coverage masks
};

int pmh_build_slabs(pmh_polys P, cudaStream_t s);
int pmh_launch_slabs_fixed(pmh_ctx ctx, const int2* xy, const int64_t* off, int64_t max_polys,
                           const int64_t* d_n, SlabInfo* info, int64_t* sizes, int64_t* sums,
                           int32_t* slab_ptr, int64_t cap_ptr, int32_t* cursor, int32_t* slab_edges,
                           int64_t cap_edges, cudaStream_t s);
int pmh_build_masks(pmh_polys P, cudaStream_t s);

// coverage masks (masks.cu): 16 x 16 cells of 2^cwl x 2^chl lattice units over the
// clipped bounding box; 2 bits per cell (0 outside, 1 inside, 2 boundary)
constexpr int kMaskMaxVerts = 256;
__host__ __device__ __forceinline__ int mask_cell_log2(int w)
{
    int a = (w + 15) >> 4, l = 0;
    while ((1 << l) < a) ++l;
    return l;
}
int pmh_build_cost_order(pmh_polys P, cudaStream_t s);   // P->order (walk form without the index)
int pmh_build_class_order(pmh_polys P, cudaStream_t s);  // P->order_cls and the class counts

struct pmh_index_s {
    pmh_ctx ctx = nullptr;
    int device = 0;
    int64_t n = 0;
    pmh_params params{};
    int band_bits = 0;
    uint32_t* hashes = nullptr;     // [n][K]
    uint32_t* sorted_comp = nullptr;  // [n * bands] composite (band, key) sort keys
    int32_t* sorted_id = nullptr;     // [n * bands]
    // directory of the sorted composites: dir[s] = first entry whose composite >> dir_shift
    // is >= s, for s in [0, ceil((bands << (32 - band_bits)) / 2^dir_shift)] (a lower bound
    // of a valid composite reads one short range)
    int64_t* dir = nullptr;
    int dir_shift = 32;
};

// grow-only scratch buffer of the context
int pmh_scratch(pmh_ctx ctx, int slot, size_t bytes, void** out);
int pmh_check_params(const pmh_params* p);
int pmh_check_device(pmh_ctx ctx);

// ---------------------------------------------------------------------------
// Stream points (SplitMix64, Steele/Lea/Flood 2014)
// ---------------------------------------------------------------------------
#define PMH_GAMMA 0x9E3779B97F4A7C15ull
#define PMH_M1 0xBF58476D1CE4E5B9ull
#define PMH_M2 0x94D049BB133111EBull

__host__ __device__ __forceinline__ uint64_t pmh_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * PMH_M1;
    z = (z ^ (z >> 27)) * PMH_M2;
    return z ^ (z >> 31);
}

// low 32 bits of the mix: all a lattice point needs (x = bits 0..15, y = 16..31)
__device__ __forceinline__ uint32_t pmh_mix64_lo(uint64_t z)
{
    z = (z ^ (z >> 30)) * PMH_M1;
    z = (z ^ (z >> 27)) * PMH_M2;
    return (uint32_t)(z ^ (z >> 31));
}

// ---------------------------------------------------------------------------
// Scans (scan.cu)
// ---------------------------------------------------------------------------
// exclusive prefix sum of n int64 values in place-able form: out[i] = sum in[0..i-1],
// out[n] = total (out has n + 1 entries).  in may alias out.
// sums_buffer (optional, pmh_scan_sums_size(n) entries) replaces the context scratch,
// so that a captured graph owns every buffer it touches.
int pmh_exclusive_scan_i64(pmh_ctx ctx, const int64_t* in, int64_t* out, int64_t n,
                           cudaStream_t s, int64_t* sums_buffer = nullptr);
int64_t pmh_scan_sums_size(int64_t n);

// ---------------------------------------------------------------------------
// Internal launchers shared by the public calls and the captured query graph.
// d_n (optional): device-side count that caps the launch-time size n, so a graph
// captured for a maximum batch serves any smaller batch.  d_flags (optional):
// device status word; bits 0-2 = invalid polygons (set by prep: 1 offsets,
// 2 fewer than 3 vertices, 4 coordinate range), bit 3 = candidate overflow (set
// by the join).  Kernels after a failed stage do nothing.
// ---------------------------------------------------------------------------
int pmh_launch_prep(int sm_count, const int2* xy, const int64_t* off, int64_t n_polys,
                    const int64_t* d_n, int64_t n_vertices, int4* bbox, int64_t* area2,
                    int* status, cudaStream_t s);
int pmh_launch_sign(pmh_ctx ctx, const int2* xy, const int64_t* off, const int4* bbox,
                    const SlabInfo* slabs, const int32_t* slab_ptr, const int32_t* slab_edges,
                    const int32_t* order, const pmh_params* P, int64_t n_polys,
                    const int64_t* d_n, const int* d_flags, unsigned long long* ticket,
                    uint32_t* out, cudaStream_t s, const int64_t* area2 = nullptr,
                    const StreamIndexView* sidx = nullptr, const uint32_t* masks = nullptr,
                    const int32_t* order_cls = nullptr, int64_t n_indexed = 0,
                    int64_t n_whole_cost = 0);
// every polygon in one persistent launch (sign_unified.cu): slots list[0 ..
// n_slots) (list nullptr: slot = polygon id), the first n_chunked as (polygon,
// 32-hash chunk) items, the rest whole; d_n (optional) caps n_slots on the
// device, d_flags (optional) skips a batch that failed validation; U = points
// per lane per round of the walk form (2, 4 or 8); work (optional) the six
// work counters.  The last n_indexed_tail slots of a class list (staged polygons
// of the indexed form, the class order's last class) get a launch of their own
// through a build of the kernel without the other paths.
int pmh_launch_sign_unified(pmh_ctx ctx, int U, const int2* xy, const int64_t* off,
                            const int4* bbox, const int64_t* area2, const SlabInfo* slabs,
                            const int32_t* slab_ptr, const int32_t* slab_edges, const int32_t* list,
                            int64_t n_slots, int64_t n_chunked, int64_t n_indexed_tail,
                            const int64_t* d_n, const int* d_flags, const pmh_params* P,
                            const StreamIndexView& S, unsigned long long* ticket, uint32_t* out,
                            unsigned long long* work, cudaStream_t s);
// bucket join (lsh.cu): the count pass (write false: counts) or the fill pass (write
// true: the CSR rows).  `stage` (nullable, pmh_join_stage_bytes(Q, pool_ints) bytes,
// the same buffer for both passes, 16-byte aligned) lets the count pass keep the rows
// it sorted, up to pool_ints ids in all, so that the fill pass copies them; the fill
// pass of a call whose count pass had no stage gets none either
size_t pmh_join_stage_bytes(int64_t Q, int64_t pool_ints);
int pmh_launch_query(pmh_index X, const uint32_t* qh, int64_t Q, const int64_t* d_n,
                     int64_t* counts, const int64_t* row_ptr, int32_t* cand, int64_t cap,
                     void* stage, int64_t pool_ints, int* d_flags, bool write, cudaStream_t s);
int pmh_launch_agree(pmh_ctx ctx, const uint32_t* qh, const uint32_t* ph, const int64_t* row_ptr,
                     const int32_t* cand, int64_t Q, int64_t cap, const pmh_params* P,
                     uint16_t* count, uint32_t* bandmask, const int* d_flags, cudaStream_t s);
// per-set inputs of the reranker's features: log features, boxes and twice the areas
struct FeatSrc {
    const float2* feat;
    const int4* bbox;
    const int64_t* area2;
};

// a pair's per-polygon inputs of its feature row
struct FeatPair {
    float2 qf, pf;       // (log2 area / 32, log2 vertex count / 16)
    int4 qb, pb;         // bounding boxes
    long long qa2, pa2;  // twice the signed areas
};
__device__ __forceinline__ FeatPair pmh_feat_pair(const FeatSrc& qf, const FeatSrc& pf, int64_t q, int64_t p)
{
    return FeatPair{qf.feat[q], pf.feat[p], qf.bbox[q], pf.bbox[p], qf.area2[q], pf.area2[p]};
}

// Column 32 + col (col < 16) of the reranker's feature row of a pair (A7) from its
// comparison counts over the K hashes -- c equal (and not the sentinel), lt / gt
// lower / higher than the candidate's -- and the two polygons' inputs; 40..47 are
// zero.  Every kernel that writes feature rows takes these values from here, so all
// feed the network the same bf16 values.
__device__ __forceinline__ float pmh_feature_col(int col, int K, int c, int lt, int gt, const FeatPair& in)
{
    switch (col) {
    case 0: return (float)c / (float)K;
    case 1: return in.qf.x;
    case 2: return in.pf.x;
    case 3: return in.qf.y;
    case 4: return in.pf.y;
    case 5: return (float)lt / (float)K;
    case 6: return (float)gt / (float)K;
    case 7: {
        // upper bound of J: the intersection is at most min(|q|, |p|, overlap of the
        // two bounding boxes)
        const int4 qb = in.qb, pb = in.pb;
        const float ow = (float)max(0, min(qb.z, pb.z) - max(qb.x, pb.x));
        const float oh = (float)max(0, min(qb.w, pb.w) - max(qb.y, pb.y));
        const long long qa = in.qa2, pa = in.pa2;
        const float a = 0.5f * (float)(qa < 0 ? -qa : qa);
        const float bq = 0.5f * (float)(pa < 0 ? -pa : pa);
        const float mn = fminf(fminf(a, bq), ow * oh);
        const float den = a + bq - mn;
        return den > 0.f ? mn / den : 0.f;
    }
    default: return 0.f;
    }
}

// The feature row of a pair, one warp per pair: eq = K / 32 equality words (bit
// k % 32 of word k / 32 set iff h_k(q) = h_k(p) != T).  Lane l returns column l
// (all K / 32 hashes of group l equal) in lo and, for l < 16, column 32 + l in hi.
__device__ __forceinline__ void pmh_feature_values(const uint32_t* eq, int K, int c, int lt, int gt,
                                                   const FeatPair& in, int lane, float& lo, float& hi)
{
    const int g = K / 32;
    bool all = true;
    for (int t = 0; t < g && all; ++t) {
        const int k = lane * g + t;
        all = (eq[k >> 5] >> (k & 31)) & 1u;
    }
    lo = all ? 1.f : 0.f;
    hi = pmh_feature_col(lane, K, c, lt, gt, in);
}
int pmh_launch_agree_features(pmh_ctx ctx, const uint32_t* qh, const uint32_t* ph,
                              const int64_t* row_ptr, const int32_t* cand, int64_t Q, int64_t cap,
                              const pmh_params* P, uint16_t* count, uint32_t* bandmask,
                              uint16_t* feat, FeatSrc qf, FeatSrc pf, const int* d_flags,
                              cudaStream_t s);
// exact refinement of fixed-width top-m lists (ids [Q][m], nlist [Q]) to the top-k by
// (J desc, id asc) (refine.cu); jv: Q * m doubles of scratch; ticket: the grid's counter;
// d_n (optional) caps Q on the device
int pmh_launch_refine_topk(pmh_ctx ctx, const int2* qxy, const int64_t* qoff, const int64_t* qarea2,
                           const int4* qbox, pmh_polys db, const int32_t* ids, const int32_t* nlist, int64_t Q,
                           const int64_t* d_n, int32_t m, int32_t k, double* jv,
                           unsigned long long* ticket, int32_t* top_ids, double* top_j,
                           cudaStream_t s);
// fixed-width lists ids [Q][m] with counts n [Q] to compact CSR (row_ptr [Q + 1], cand);
// rows at or past *d_q (optional) are empty; counts: Q entries of scratch; sums: the
// scan's partial sums (pmh_scan_sums_size(Q) entries; nullptr: context scratch)
int pmh_launch_lists_to_csr(pmh_ctx ctx, const int32_t* ids, const int32_t* n, int64_t Q, int32_t m,
                            const int64_t* d_q, int64_t* counts, int64_t* sums, int64_t* row_ptr,
                            int32_t* cand, cudaStream_t s);
// per-polygon reranker inputs (log2 area / 32, log2 vertex count / 16) of polygons
// [0, n) (capped by *d_n when given)
int pmh_launch_poly_feat(int sm_count, const int64_t* area2, const int64_t* off, int64_t n,
                         const int64_t* d_n, float2* out, cudaStream_t s);
// reranker scores of n feature rows (rerank.cu)
int pmh_launch_rerank_forward(pmh_rerank r, const uint16_t* feat, int64_t n_rows, float* score,
                              int* d_flags, cudaStream_t s);
// the learned form's features, scores and top-m in one launch (rerank.cu): shortlist
// ids [Q][S] / counts n[Q] (top-S by count) to ids [Q][m] (-1 padded) and counts
// [Q] by (predicted Jaccard desc, id asc); S must divide 128 (S >= 4), K % 32 == 0
bool pmh_rerank_select_fits(int S, int K);
int pmh_launch_rerank_select(pmh_rerank r, const uint32_t* qh, const uint32_t* ph, const int32_t* sl_ids,
                             const int32_t* sl_n, int64_t Q, const int64_t* d_n, int S, int m,
                             const pmh_params* P, FeatSrc qf, FeatSrc pf, int32_t* out_ids, int32_t* out_n,
                             int* d_flags, cudaStream_t s);
// top-m per row (estimate.cu); K bounds the counts (0: up to 4,096)
int pmh_launch_topm(const int64_t* row_ptr, const int32_t* cand, const uint16_t* count,
                    const float* score, int64_t Q, int32_t m, int K, int32_t* out_ids, int32_t* out_n,
                    const int* d_flags, cudaStream_t s);

// signing kernel variants (points per lane per round x warps per block)
int pmh_sign_variant_count();
void pmh_sign_variant_shape(int v, int* points_per_lane, int* warps);

// stable LSD radix sort of (uint32 key, int32 value) pairs; result in keys/vals.
int pmh_radix_sort_u32(pmh_ctx ctx, uint32_t* keys, int32_t* vals, int64_t n, int key_bits,
                       cudaStream_t s);

// warp helpers
__device__ __forceinline__ unsigned pmh_lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

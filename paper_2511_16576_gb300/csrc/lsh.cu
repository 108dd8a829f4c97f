// lsh.cu -- steps A2 (band keys), A3 (bucket index) and A4 (bucket join).
//
// The paper inserts every polygon into a hashmap keyed on its MinHash code and
// takes the bucket members as refinement candidates (Sec. 3.2 after Theorem 1,
// Sec. 5.2; "2 hashmaps", Sec. 5.3).  Here one hashmap per band is a sorted
// array: entry (band j, polygon p) gets a 32-bit composite sort key
// (j in the top band_bits bits, the top bits of the 64-bit band key below),
// stable-radix-sorted so that equal composites keep ascending ids.  A
// directory over the composites' top bits (about eight entries per slot)
// bounds each lookup to one short range.  A query
// binary-searches its composite there per band and walks the equal range, keeping
// the entries whose r-tuple equals its own (exact bucket membership; an entry of
// another key shares the composite with probability ~n / 2^(32 - band_bits) per
// lookup and costs one tuple read).  The per-band id lists are ascending, so a
// warp merges them (min over lanes) into the sorted, duplicate-free candidate row.
#include <algorithm>

#include "pmh_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t band_key(const uint32_t* __restrict__ h, int j, int rows,
                                             uint32_t T, uint64_t lsh_seed)
{
    uint64_t a = pmh_mix64(lsh_seed + (uint64_t)(j + 1) * PMH_GAMMA);
    bool valid = true;
    for (int t = 0; t < rows; ++t) {
        uint32_t v = h[j * rows + t];
        valid &= v != T;
        a = pmh_mix64(a ^ (uint64_t)v);
    }
    if (a == PMH_INVALID_KEY) a = PMH_INVALID_KEY - 1;
    return valid ? a : PMH_INVALID_KEY;
}

__global__ void band_key_kernel(const uint32_t* __restrict__ hashes, int64_t n, int K, int bands,
                                int rows, uint32_t T, uint64_t lsh_seed, uint64_t* __restrict__ keys)
{
    int64_t total = n * bands;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = t / bands;
        int j = (int)(t - p * bands);
        keys[t] = band_key(hashes + p * K, j, rows, T, lsh_seed);
    }
}

__device__ __forceinline__ uint32_t composite(uint64_t key, int j, int band_bits)
{
    if (key == PMH_INVALID_KEY) return 0xFFFFFFFFu;
    return ((uint32_t)j << (32 - band_bits)) | (uint32_t)(key >> (32 + band_bits));
}

// entries in polygon-major order, e = p * bands + j (within one band, ascending ids:
// the stable sort keeps them ascending inside a bucket), band keys computed from the
// hashes in place
__global__ void fill_entries_kernel(const uint32_t* __restrict__ hashes, int64_t n, int K, int bands,
                                    int rows, uint32_t T, uint64_t lsh_seed, int band_bits,
                                    uint32_t* __restrict__ comp, int32_t* __restrict__ ids)
{
    const int64_t total = n * bands;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bands;
        const int j = (int)(e - p * bands);
        comp[e] = composite(band_key(hashes + p * K, j, rows, T, lsh_seed), j, band_bits);
        ids[e] = (int32_t)p;
    }
}

// The directory covers the composites of valid entries, [0, cmax) with
// cmax = bands << (32 - band_bits) (invalid entries, all ones, sort last and are
// never looked up): dir[s] = first sorted entry whose composite >> sh is >= s,
// for s in [0, ceil(cmax / 2^sh)].  Thread e writes the slots after its predecessor's,
// up to its own (thread m: up to the last), so every slot is written once; the
// keys are uniform, so gaps are a slot or two (a band without one valid entry
// leaves one thread a gap of 2^(32 - band_bits - sh) slots).
__global__ void dir_kernel(const uint32_t* __restrict__ comp, int64_t m, int sh, int64_t cmax,
                           int64_t* __restrict__ dir)
{
    const int64_t top = (cmax + (1ll << sh) - 1) >> sh;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cs = e < m ? min((int64_t)comp[e], cmax) >> sh : top;
        const int64_t ps = e == 0 ? 0 : (min((int64_t)comp[e - 1], cmax) >> sh) + 1;
        for (int64_t s = ps; s <= cs; ++s) dir[s] = e;
    }
}

// first sorted entry whose composite is >= c
__device__ __forceinline__ int64_t comp_lower_bound(const uint32_t* __restrict__ comp,
                                                    const int64_t* __restrict__ dir, int sh, uint32_t c)
{
    const uint32_t s = c >> sh;
    int64_t lo = dir[s], hi = dir[s + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (comp[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int kMaxBandsPerLane = 4;  // bands <= 128
constexpr int32_t kNone = 0x7FFFFFFF;

struct BandCursor {
    int64_t cur;
    uint32_t comp;
    int j;
    int32_t head;
};

__device__ __forceinline__ bool tuple_equal(const uint32_t* __restrict__ a,
                                            const uint32_t* __restrict__ b, int j, int rows)
{
    for (int t = 0; t < rows; ++t)
        if (a[j * rows + t] != b[j * rows + t]) return false;
    return true;
}

// advance c to the next entry of its band that is an exact bucket member: the
// walk reads the sorted arrays sequentially and gathers the tuple of every entry
// with the query's composite (the bucket's members, and the rare entries of other
// keys sharing the composite's key bits)
__device__ __forceinline__ void advance(BandCursor& c, const uint32_t* __restrict__ comp,
                                        const int32_t* __restrict__ ids,
                                        const uint32_t* __restrict__ dbh,
                                        const uint32_t* __restrict__ qh, int64_t m, int K,
                                        int bands, int rows)
{
    c.head = kNone;
    while (c.cur < m && comp[c.cur] == c.comp) {
        const int64_t e = c.cur++;
        const int32_t p = ids[e];
        if (tuple_equal(qh, dbh + (int64_t)p * K, c.j, rows)) {
            c.head = p;
            return;
        }
    }
}

// One warp per query.  The count pass writes the row length (0 for rows past the
// device-side batch size d_n or after a failed validation, flag bits 0-2); the
// fill pass writes the row, unless the total exceeds the capacity (then it
// raises flag bit 3).
template <bool kWrite>
__global__ void query_kernel(const uint32_t* __restrict__ qhashes, int64_t Q, int K, int bands,
                             int rows, uint32_t T, uint64_t lsh_seed, int band_bits,
                             const uint32_t* __restrict__ comp, const int32_t* __restrict__ ids,
                             const uint32_t* __restrict__ dbh,
                             const int64_t* __restrict__ dir, int dsh, int64_t m,
                             int64_t* __restrict__ counts,
                             const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cand,
                             int64_t cap, const int64_t* __restrict__ d_n, int* __restrict__ d_flags)
{
    const int lane = threadIdx.x & 31;
    int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= Q) return;
    const bool skip = (d_n && q >= *d_n) || (d_flags && (*d_flags & 7));
    if (!kWrite && skip) {
        if (lane == 0) counts[q] = 0;
        return;
    }
    if (kWrite) {
        if (skip) return;
        if (row_ptr[Q] > cap) {
            if (lane == 0 && d_flags) atomicOr(d_flags, 8);
            return;
        }
    }
    const uint32_t* qh = qhashes + q * K;
    BandCursor cur[kMaxBandsPerLane];
#pragma unroll
    for (int t = 0; t < kMaxBandsPerLane; ++t) {
        int j = lane + 32 * t;
        cur[t].head = kNone;
        cur[t].j = j;
        if (j >= bands) continue;
        uint64_t key = band_key(qh, j, rows, T, lsh_seed);
        if (key == PMH_INVALID_KEY) continue;
        cur[t].comp = composite(key, j, band_bits);
        cur[t].cur = comp_lower_bound(comp, dir, dsh, cur[t].comp);
        advance(cur[t], comp, ids, dbh, qh, m, K, bands, rows);
    }
    int64_t out = kWrite ? row_ptr[q] : 0;
    int64_t cnt = 0;
    for (;;) {
        int32_t mine = kNone;
#pragma unroll
        for (int t = 0; t < kMaxBandsPerLane; ++t) mine = min(mine, cur[t].head);
        int32_t best = __reduce_min_sync(0xffffffffu, mine);
        if (best == kNone) break;
        if (kWrite && lane == 0) cand[out + cnt] = best;
        ++cnt;
#pragma unroll
        for (int t = 0; t < kMaxBandsPerLane; ++t)
            if (cur[t].head == best) advance(cur[t], comp, ids, dbh, qh, m, K, bands, rows);
    }
    if (!kWrite && lane == 0) counts[q] = cnt;
}

// Many-band join: one block per query.  Each warp takes one band at a time;
// its lanes stride over the band's bucket (coalesced reads of the sorted
// entries, the next 32 read while the current ones are checked) and insert
// exact matches into a shared-memory open-addressing set, which drops the
// duplicates (a candidate found in several bands).  The set is then compacted
// and bitonic-sorted, which yields the same ascending, duplicate-free row as the
// warp merge.  Two set sizes: the small one (8,192 slots, several blocks per SM)
// takes every row of at most 4,096 distinct candidates; a row that overflows it
// stops walking, is marked (count -1) and counted again, like every longer row
// filled, by the large one (32,768 slots, one block of 1,024 threads per SM).
// A row beyond even that falls back to the warp merge (warp 0).  With a staging
// pool, the count pass also writes each sorted row there (a slice reserved by an
// atomic cursor; a row that no longer fits is left unstaged) and the fill pass
// copies the staged rows into place (copy_rows_kernel) and joins only the rest.
template <bool kBig>
struct JoinShape {
    static constexpr int kThreads = kBig ? 1024 : 256;
    static constexpr int kLog2Table = kBig ? 15 : 13;
    static constexpr int kTable = 1 << kLog2Table;   // shared set slots
    static constexpr int kMaxUnique = kTable / 2;    // load factor <= 1/2
    static constexpr size_t kSmem = sizeof(int32_t) * (kTable + kMaxUnique);
};
constexpr int kSmallRowMax = JoinShape<false>::kMaxUnique;

// where the count pass leaves its sorted rows: pool slices handed out by cursor;
// where[q] = offset of row q's slice, -1 if the row is not staged
struct JoinStage {
    int32_t* pool = nullptr;
    int64_t pool_ints = 0;
    unsigned long long* cursor = nullptr;  // [0]: pool ids handed out, [1]: large-set row ticket
    int64_t* where = nullptr;
};

__device__ int64_t merge_row(const uint32_t* __restrict__ qh, int K, int bands, int rows, uint32_t T,
                             uint64_t lsh_seed, int band_bits, const uint32_t* __restrict__ comp,
                             const int32_t* __restrict__ ids, const uint32_t* __restrict__ dbh, const int64_t* __restrict__ dir,
                             int dsh, int64_t m, int32_t* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    BandCursor cur[kMaxBandsPerLane];
#pragma unroll
    for (int t = 0; t < kMaxBandsPerLane; ++t) {
        int j = lane + 32 * t;
        cur[t].head = kNone;
        cur[t].j = j;
        if (j >= bands) continue;
        uint64_t key = band_key(qh, j, rows, T, lsh_seed);
        if (key == PMH_INVALID_KEY) continue;
        cur[t].comp = composite(key, j, band_bits);
        cur[t].cur = comp_lower_bound(comp, dir, dsh, cur[t].comp);
        advance(cur[t], comp, ids, dbh, qh, m, K, bands, rows);
    }
    int64_t cnt = 0;
    for (;;) {
        int32_t mine = kNone;
#pragma unroll
        for (int t = 0; t < kMaxBandsPerLane; ++t) mine = min(mine, cur[t].head);
        int32_t best = __reduce_min_sync(0xffffffffu, mine);
        if (best == kNone) break;
        if (out && lane == 0) out[cnt] = best;
        ++cnt;
#pragma unroll
        for (int t = 0; t < kMaxBandsPerLane; ++t)
            if (cur[t].head == best) advance(cur[t], comp, ids, dbh, qh, m, K, bands, rows);
    }
    return cnt;
}

template <int kLog2>
__device__ __forceinline__ uint32_t slot_hash(int32_t p)
{
    return ((uint32_t)p * 0x9E3779B1u) >> (32 - kLog2);
}

// candidate p's tuple of band j equals the query's, both tuples read at once (16-byte
// loads for 4 or 8 rows when vec: K % 4 == 0)
__device__ __forceinline__ bool tuple_match2(const uint32_t* __restrict__ qh, const uint32_t* __restrict__ dbrow,
                                             int j, int rows, bool vec)
{
    const uint32_t* a = qh + j * rows;
    const uint32_t* b = dbrow + j * rows;
    if (vec && rows == 4) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(a)), v = __ldg(reinterpret_cast<const uint4*>(b));
        return u.x == v.x && u.y == v.y && u.z == v.z && u.w == v.w;
    }
    if (vec && rows == 8) {
        const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(a)), v0 = __ldg(reinterpret_cast<const uint4*>(b));
        const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(a) + 1), v1 = __ldg(reinterpret_cast<const uint4*>(b) + 1);
        return u0.x == v0.x && u0.y == v0.y && u0.z == v0.z && u0.w == v0.w && u1.x == v1.x && u1.y == v1.y &&
               u1.z == v1.z && u1.w == v1.w;
    }
    if (rows <= 8) {
        uint32_t u[8], v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            u[t] = t < rows ? __ldg(a + t) : 0u;
            v[t] = t < rows ? __ldg(b + t) : 0u;
        }
        bool eq = true;
#pragma unroll
        for (int t = 0; t < 8; ++t) eq &= u[t] == v[t];
        return eq;
    }
    return tuple_equal(qh, dbrow, j, rows);
}

// per-band state of a block's walk (bands <= 128)
struct JoinBands {
    int64_t lo[kMaxBandsPerLane * 32];   // first entry of the band's composite
    int64_t off[kMaxBandsPerLane * 32 + 1];  // prefix of the bands' entry counts
};

// The set's walk over the query's bands, keeping the exact bucket members with ids in
// [id_lo, id_hi); returns the number of distinct ids inserted (more than kMaxUnique:
// the walk stopped early).  The equal-composite range of every band is found first
// (a thread per band: two directory lookups); the ranges' entries, concatenated, are
// then split evenly over the block's warps, 32 consecutive entries at a time, two
// chunks in flight per warp -- one band's bucket of thousands of entries no longer
// keeps one warp busy while the others wait.  Block-wide; starts and ends with a
// barrier.
template <bool kBig>
__device__ int join_walk(const uint32_t* __restrict__ qh, int K, int bands, int rows, uint32_t T,
                         uint64_t lsh_seed, int band_bits, const uint32_t* __restrict__ comp,
                         const int32_t* __restrict__ ids, const uint32_t* __restrict__ dbh,
                         const int64_t* __restrict__ dir, int dsh, int64_t m, int32_t id_lo, int32_t id_hi,
                         int32_t* table, int* n_unique, JoinBands& jb)
{
    using S = JoinShape<kBig>;
    constexpr int kJoinTable = S::kTable, kJoinMaxUnique = S::kMaxUnique;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    volatile int* nu_v = n_unique;
    const bool vec = (K & 3) == 0;
    __syncthreads();
    for (int i = threadIdx.x; i < kJoinTable; i += blockDim.x) table[i] = kNone;
    if (threadIdx.x == 0) *n_unique = 0;
    for (int j = threadIdx.x; j < bands; j += blockDim.x) {
        const uint64_t key = band_key(qh, j, rows, T, lsh_seed);
        int64_t lo = 0, n = 0;
        if (key != PMH_INVALID_KEY) {
            const uint32_t c = composite(key, j, band_bits);
            lo = comp_lower_bound(comp, dir, dsh, c);
            const int64_t hi = c == 0xFFFFFFFFu ? m : comp_lower_bound(comp, dir, dsh, c + 1);
            n = hi - lo;
        }
        jb.lo[j] = lo;
        jb.off[j + 1] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        jb.off[0] = 0;
        for (int j = 0; j < bands; ++j) {
            acc += jb.off[j + 1];
            jb.off[j + 1] = acc;
        }
    }
    __syncthreads();
    const int64_t total = jb.off[bands];
    for (int64_t g0 = (int64_t)wid * 64; g0 < total; g0 += (int64_t)nw * 64) {
        if (__shfl_sync(0xffffffffu, *nu_v, 0) > kJoinMaxUnique) break;  // falls back anyway
        // two chunks of 32 entries: each lane's band by bisection over the prefix
        int jj[2];
        int32_t pp[2];
        bool in[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t g = g0 + 32 * u + lane;
            in[u] = g < total;
            int lo = 0, hi = bands;  // last j with off[j] <= g
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (jb.off[mid] <= g) lo = mid;
                else hi = mid;
            }
            jj[u] = lo;
            pp[u] = in[u] ? ids[jb.lo[lo] + (g - jb.off[lo])] : 0;
        }
        int added = 0;  // the warp's new ids, added to the set's count once per chunk pair
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int32_t pe = pp[u];
            if (in[u] && pe >= id_lo && pe < id_hi && tuple_match2(qh, dbh + (int64_t)pe * K, jj[u], rows, vec)) {
                uint32_t h = slot_hash<S::kLog2Table>(pe);
                for (int probe = 0; probe < kJoinTable; ++probe, h = (h + 1) & (kJoinTable - 1)) {
                    const int32_t old = atomicCAS(&table[h], kNone, pe);
                    if (old == kNone) {
                        ++added;
                        break;
                    }
                    if (old == pe) break;
                    if (*nu_v > kJoinMaxUnique) break;  // the set falls back anyway
                }
            }
        }
        added = __reduce_add_sync(0xffffffffu, added);
        if (lane == 0 && added) atomicAdd(n_unique, added);
    }
    __syncthreads();
    return *n_unique;
}

// the set's nu ids, ascending, to out (compaction by a block scan over contiguous
// slot ranges into buf, then a bitonic sort of the next power of two above nu)
template <bool kBig>
__device__ void join_emit(int32_t* table, int nu, int* wsum, int32_t* __restrict__ out)
{
    using S = JoinShape<kBig>;
    constexpr int kJoinTable = S::kTable;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t* buf = table + kJoinTable;
    constexpr int kPer = kJoinTable / S::kThreads;
    const int s0 = threadIdx.x * kPer;
    int mine = 0;
    for (int i = 0; i < kPer; ++i) mine += table[s0 + i] != kNone;
    int x = mine;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int pos = x - mine;
    for (int w = 0; w < wid; ++w) pos += wsum[w];
    for (int i = 0; i < kPer; ++i)
        if (table[s0 + i] != kNone) buf[pos++] = table[s0 + i];
    int n2 = 1;
    while (n2 < nu) n2 <<= 1;
    for (int i = nu + threadIdx.x; i < n2; i += blockDim.x) buf[i] = kNone;
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ jj;
                if (l > i) {
                    const int32_t a = buf[i], b = buf[l];
                    if ((a > b) == ((i & k) == 0)) {
                        buf[i] = b;
                        buf[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < nu; i += blockDim.x) out[i] = buf[i];
    __syncthreads();
}

// A row of more distinct candidates than the large set holds is joined in id-range
// passes: pass r keeps the ids in [r N / P, (r + 1) N / P), so the passes' sorted
// outputs concatenate to the sorted row; P doubles until every pass fits (beyond
// kMaxPasses the row takes the warp merge).  Such rows are not staged: the count
// pass records -P in where[q] (-2 kMaxPasses for a merged row) and the fill pass
// joins them again the same way.
constexpr int kMaxPasses = 64;

template <bool kWrite, bool kBig>
__global__ void __launch_bounds__(JoinShape<kBig>::kThreads)
join_kernel(const uint32_t* __restrict__ qhashes, int64_t Q, int K, int bands, int rows, uint32_t T,
            uint64_t lsh_seed, int band_bits, const uint32_t* __restrict__ comp,
            const int32_t* __restrict__ ids, const uint32_t* __restrict__ dbh,
            const int64_t* __restrict__ dir, int dsh, int64_t m, int64_t n_db, int64_t* __restrict__ counts,
            const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cand, int64_t cap,
            JoinStage st, const int64_t* __restrict__ d_n, int* __restrict__ d_flags)
{
    using S = JoinShape<kBig>;
    constexpr int kJoinMaxUnique = S::kMaxUnique;
    extern __shared__ int32_t table[];  // kJoinTable slots, then kJoinMaxUnique sorted ids
    __shared__ int n_unique;
    __shared__ long long stage_off;
    __shared__ int wsum[S::kThreads / 32];
    __shared__ JoinBands jb;
    __shared__ long long next_q;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the large set's count pass takes rows from a ticket (its rows' sizes vary several
    // times over); the other passes step through the rows
    unsigned long long* ticket = (!kWrite && kBig && st.cursor) ? st.cursor + 1 : nullptr;
    for (int64_t q = blockIdx.x;; q += gridDim.x) {
        if (ticket) {
            __syncthreads();
            if (threadIdx.x == 0) next_q = (long long)atomicAdd(ticket, 1ull);
            __syncthreads();
            q = next_q;
        }
        if (q >= Q) break;
        const bool skip = (d_n && q >= *d_n) || (d_flags && (*d_flags & 7));
        if (skip) {
            if (!kWrite && !kBig && threadIdx.x == 0) {
                counts[q] = 0;
                if (st.where) st.where[q] = -1;
            }
            continue;
        }
        if (kWrite && row_ptr[Q] > cap) {
            if (threadIdx.x == 0 && d_flags) atomicOr(d_flags, 8);
            return;
        }
        // rows by size: the small set counts every row and fills the short ones; the
        // large set counts the rows that overflowed the small one and fills the long ones;
        // staged rows are copied instead
        if (!kWrite && kBig && counts[q] >= 0) continue;
        if (kWrite && ((row_ptr[q + 1] - row_ptr[q] > kSmallRowMax) != kBig)) continue;
        int passes = 1;
        if (kWrite && st.where) {
            const int64_t w = st.where[q];
            if (w >= 0) continue;
            passes = (int)max((int64_t)1, -w);
        }
        const uint32_t* qh = qhashes + q * K;
        int64_t total = 0;
        bool merged = passes > kMaxPasses;
        while (!merged) {  // passes over id ranges (one, unless the row overflows the large set)
            bool over = false;
            total = 0;
            for (int r = 0; r < passes; ++r) {
                const int32_t lo = (int32_t)(n_db * r / passes), hi = (int32_t)(n_db * (r + 1) / passes);
                const int nu = join_walk<kBig>(qh, K, bands, rows, T, lsh_seed, band_bits, comp, ids, dbh, dir,
                                               dsh, m, lo, hi, table, &n_unique, jb);
                if (nu > kJoinMaxUnique) {
                    over = true;
                    break;
                }
                int32_t* out = nullptr;
                if (kWrite) {
                    out = cand + row_ptr[q] + total;
                } else if (passes == 1) {
                    // the count pass stages a one-pass row when the pool has room
                    if (threadIdx.x == 0) {
                        long long off = -1;
                        if (st.pool && st.where) {
                            const unsigned long long o = atomicAdd(st.cursor, (unsigned long long)nu);
                            if ((long long)(o + (unsigned long long)nu) <= st.pool_ints) off = (long long)o;
                        }
                        stage_off = off;
                    }
                    __syncthreads();
                    if (stage_off >= 0) out = st.pool + stage_off;
                }
                if (out) join_emit<kBig>(table, nu, wsum, out);
                total += nu;
            }
            if (!over) break;
            if (!kBig) break;  // the large set takes the row
            passes *= 2;
            if (passes > kMaxPasses) {
                merged = true;
                break;
            }
        }
        if (!kBig && n_unique > kJoinMaxUnique) {
            // the small set overflowed: the large set counts this row again
            if (threadIdx.x == 0) {
                counts[q] = -1;
                if (st.where) st.where[q] = -1;
            }
            continue;
        }
        if (merged) {  // beyond the id-range passes: merge the row with warp 0 (never staged)
            if (wid == 0) {
                const int64_t cnt = merge_row(qh, K, bands, rows, T, lsh_seed, band_bits, comp, ids, dbh, dir,
                                              dsh, m, kWrite ? cand + row_ptr[q] : nullptr);
                if (!kWrite && lane == 0) {
                    counts[q] = cnt;
                    if (st.where) st.where[q] = -2 * (int64_t)kMaxPasses;
                }
            }
            continue;
        }
        if (!kWrite && threadIdx.x == 0) {
            counts[q] = total;
            if (st.where) st.where[q] = passes > 1 ? -(int64_t)passes : (long long)stage_off;
        }
    }
}

// fill pass of the staged rows: a block per row copies its pool slice into place
// (four independent loads per thread in flight)
__global__ void __launch_bounds__(256)
copy_rows_kernel(JoinStage st, int64_t Q, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cand,
                 int64_t cap, const int64_t* __restrict__ d_n, int* __restrict__ d_flags)
{
    if (d_flags && (*d_flags & 7)) return;
    if (row_ptr[Q] > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && d_flags) atomicOr(d_flags, 8);
        return;
    }
    const int64_t live = d_n ? min(Q, *d_n) : Q;
    for (int64_t q = blockIdx.x; q < live; q += gridDim.x) {
        const int64_t off = st.where[q];
        if (off < 0) continue;
        const int64_t b = row_ptr[q], len = row_ptr[q + 1] - b;
        const int32_t* src = st.pool + off;
        int32_t* dst = cand + b;
        for (int64_t i = threadIdx.x; i < len; i += 4 * blockDim.x) {
            int32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = i + (int64_t)u * blockDim.x;
                v[u] = k < len ? src[k] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = i + (int64_t)u * blockDim.x;
                if (k < len) dst[k] = v[u];
            }
        }
    }
}

}  // namespace

extern "C" int pmh_band_keys(pmh_ctx ctx, const uint32_t* d_hashes, int64_t n,
                             const pmh_params* params, uint64_t* d_keys, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (n < 0 || (n > 0 && (!d_hashes || !d_keys))) return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    if (n == 0) return PMH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t total = n * params->bands;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->sm_count * 32);
    band_key_kernel<<<blocks, 256, 0, s>>>(d_hashes, n, (int)params->K, (int)params->bands,
                                           (int)params->rows, params->T, params->lsh_seed, d_keys);
    PMH_LAUNCHED("band_key_kernel");
    return PMH_OK;
}

// end of the composites of valid entries (the directory's range), and the directory's
// length (slots + 1)
static int64_t dir_cmax(pmh_index X)
{
    return (int64_t)X->params.bands << (32 - X->band_bits);
}
static size_t dir_len(pmh_index X)
{
    return (size_t)((dir_cmax(X) + (1ll << X->dir_shift) - 1) >> X->dir_shift) + 1;
}

// hashes copied in, band keys, (band, key) entries radix-sorted with ids, full keys gathered
static int index_fill(pmh_ctx ctx, pmh_index X, const uint32_t* d_hashes, cudaStream_t s)
{
    const int64_t n = X->n;
    const pmh_params* params = &X->params;
    const int bb = X->band_bits;
    const int64_t entries = n * params->bands;
    if (n == 0) {
        PMH_CUDA_TRY(cudaMemsetAsync(X->dir, 0, sizeof(int64_t) * dir_len(X), s));
        return PMH_OK;
    }
    cudaError_t e = cudaMemcpyAsync(X->hashes, d_hashes, sizeof(uint32_t) * n * params->K,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return pmh_set_error(PMH_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    int blocks = (int)std::min<int64_t>((entries + 255) / 256, (int64_t)ctx->sm_count * 32);
    fill_entries_kernel<<<blocks, 256, 0, s>>>(X->hashes, n, (int)params->K, (int)params->bands,
                                                (int)params->rows, params->T, params->lsh_seed, bb,
                                                X->sorted_comp, X->sorted_id);
    PMH_LAUNCHED("fill_entries_kernel");
    PMH_TRY(pmh_radix_sort_u32(ctx, X->sorted_comp, X->sorted_id, entries, 32, s));
    const int dblocks = (int)std::min<int64_t>((entries + 256) / 256, (int64_t)ctx->sm_count * 32);
    dir_kernel<<<dblocks, 256, 0, s>>>(X->sorted_comp, entries, X->dir_shift, dir_cmax(X), X->dir);
    PMH_LAUNCHED("dir_kernel");
    return PMH_OK;
}

// directory shift: about eight sorted entries per slot over [0, cmax), at most 2^24 slots
static int dir_shift_for(int64_t entries, int64_t cmax)
{
    int sh = 31;
    while (sh > 0 && (cmax >> (sh - 1)) <= (int64_t)1 << 24 && (cmax >> (sh - 1)) * 8 <= entries) --sh;
    return sh;
}

extern "C" int pmh_lsh_build(pmh_ctx ctx, const uint32_t* d_hashes, int64_t n,
                             const pmh_params* params, pmh_index* out, void* stream)
{
    if (!out) return pmh_set_error(PMH_ERR_ARG, "null out");
    *out = nullptr;
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (n < 0 || n >= (1ll << 31) || (n > 0 && !d_hashes))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (n=%lld)", (long long)n);
    cudaStream_t s = (cudaStream_t)stream;
    pmh_index X = new pmh_index_s();
    X->ctx = ctx;
    X->device = ctx->device;
    X->n = n;
    X->params = *params;
    int bb = 1;
    while ((1u << bb) - 1 < params->bands) ++bb;  // band index < 2^bb - 1: comp never all ones
    X->band_bits = bb;
    const int64_t entries = n * params->bands;
    X->dir_shift = dir_shift_for(entries, dir_cmax(X));
    const size_t nn = (size_t)std::max<int64_t>(n, 1), ne = (size_t)std::max<int64_t>(entries, 1);
    if (cudaMalloc(&X->hashes, sizeof(uint32_t) * nn * params->K) != cudaSuccess ||
        cudaMalloc(&X->sorted_comp, sizeof(uint32_t) * ne) != cudaSuccess ||
        cudaMalloc(&X->sorted_id, sizeof(int32_t) * ne) != cudaSuccess ||
        cudaMalloc(&X->dir, sizeof(int64_t) * dir_len(X)) != cudaSuccess) {
        cudaGetLastError();
        pmh_index_destroy(X);
        return pmh_set_error(PMH_ERR_NOMEM, "index allocation failed (n=%lld)", (long long)n);
    }
    int rc = index_fill(ctx, X, d_hashes, s);
    if (rc != PMH_OK) {
        pmh_index_destroy(X);
        return rc;
    }
    *out = X;
    return PMH_OK;
}

extern "C" int pmh_lsh_rebuild(pmh_ctx ctx, pmh_index index, const uint32_t* d_hashes, int64_t n,
                               void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!index || index->ctx != ctx || n != index->n || (n > 0 && !d_hashes))
        return pmh_set_error(PMH_ERR_ARG, "rebuild needs the index's own context and size (%lld)",
                             index ? (long long)index->n : 0ll);
    return index_fill(ctx, index, d_hashes, (cudaStream_t)stream);
}

extern "C" int pmh_index_destroy(pmh_index X)
{
    if (!X) return PMH_OK;
    cudaSetDevice(X->device);
    cudaDeviceSynchronize();
    if (X->hashes) cudaFree(X->hashes);
    if (X->sorted_comp) cudaFree(X->sorted_comp);
    if (X->sorted_id) cudaFree(X->sorted_id);
    if (X->dir) cudaFree(X->dir);
    delete X;
    return PMH_OK;
}

// one of the two block joins (both run: the large one after the small one)
template <bool kBig>
static int launch_join(pmh_index X, const uint32_t* qh, int64_t Q, const int64_t* d_n,
                       int64_t* counts, const int64_t* row_ptr, int32_t* cand, int64_t cap,
                       const JoinStage& st, int* d_flags, bool write, cudaStream_t s)
{
    using S = JoinShape<kBig>;
    const pmh_params& P = X->params;
    const int64_t m = X->n * P.bands;
    auto fn = write ? join_kernel<true, kBig> : join_kernel<false, kBig>;
    PMH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem));
    int per_sm = 1;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, S::kThreads, S::kSmem));
    const unsigned blocks =
        (unsigned)std::min<int64_t>(Q, (int64_t)X->ctx->sm_count * std::max(per_sm, 1));
    fn<<<blocks, S::kThreads, S::kSmem, s>>>(qh, Q, (int)P.K, (int)P.bands, (int)P.rows, P.T,
                                            P.lsh_seed, X->band_bits, X->sorted_comp, X->sorted_id,
                                            X->hashes, X->dir, X->dir_shift, m, X->n,
                                            write ? nullptr : counts, write ? row_ptr : nullptr,
                                            write ? cand : nullptr, write ? cap : 0, st, d_n, d_flags);
    PMH_LAUNCHED(write ? (kBig ? "join_kernel<fill,large>" : "join_kernel<fill,small>")
                       : (kBig ? "join_kernel<count,large>" : "join_kernel<count,small>"));
    return PMH_OK;
}

size_t pmh_join_stage_bytes(int64_t Q, int64_t pool_ints)
{
    return 16 + sizeof(int64_t) * (size_t)Q + sizeof(int32_t) * (size_t)pool_ints;
}

// cursor and ticket (16 bytes), where [Q], pool [pool_ints] laid out in one buffer
static JoinStage stage_view(void* buf, int64_t Q, int64_t pool_ints)
{
    JoinStage st;
    if (!buf) return st;
    char* c = static_cast<char*>(buf);
    st.cursor = reinterpret_cast<unsigned long long*>(c);
    st.where = reinterpret_cast<int64_t*>(c + 16);
    st.pool = reinterpret_cast<int32_t*>(c + 16 + sizeof(int64_t) * (size_t)Q);
    st.pool_ints = pool_ints;
    return st;
}

int pmh_launch_query(pmh_index X, const uint32_t* qh, int64_t Q, const int64_t* d_n,
                     int64_t* counts, const int64_t* row_ptr, int32_t* cand, int64_t cap,
                     void* stage, int64_t pool_ints, int* d_flags, bool write, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    const pmh_params& P = X->params;
    const int64_t m = X->n * P.bands;
    // sixteen bands or more: block per query, parallel bucket walks and a shared-memory
    // set (rows of thousands of candidates occur on dense sets; the warp merge below
    // would walk them one candidate at a time)
    if (P.bands >= 16) {
        const JoinStage st = stage_view(stage, Q, pool_ints);
        if (write) {
            if (st.where) {  // the staged rows: a copy into place
                const unsigned cblocks = (unsigned)std::min<int64_t>(Q, (int64_t)X->ctx->sm_count * 8);
                copy_rows_kernel<<<cblocks, 256, 0, s>>>(st, Q, row_ptr, cand, cap, d_n, d_flags);
                PMH_LAUNCHED("copy_rows_kernel");
            }
        } else if (st.cursor) {  // the pool cursor and the large set's row ticket
            PMH_CUDA_TRY(cudaMemsetAsync(st.cursor, 0, 2 * sizeof(unsigned long long), s));
        }
        PMH_TRY(launch_join<false>(X, qh, Q, d_n, counts, row_ptr, cand, cap, st, d_flags, write, s));
        return launch_join<true>(X, qh, Q, d_n, counts, row_ptr, cand, cap, st, d_flags, write, s);
    }
    const int wpb = 8;
    unsigned blocks = (unsigned)((Q + wpb - 1) / wpb);
    if (write) {
        query_kernel<true><<<blocks, wpb * 32, 0, s>>>(
            qh, Q, (int)P.K, (int)P.bands, (int)P.rows, P.T, P.lsh_seed, X->band_bits,
            X->sorted_comp, X->sorted_id, X->hashes, X->dir, X->dir_shift, m, nullptr,
                row_ptr, cand, cap, d_n,
            d_flags);
        PMH_LAUNCHED("query_kernel<fill>");
    } else {
        query_kernel<false><<<blocks, wpb * 32, 0, s>>>(
            qh, Q, (int)P.K, (int)P.bands, (int)P.rows, P.T, P.lsh_seed, X->band_bits,
            X->sorted_comp, X->sorted_id, X->hashes, X->dir, X->dir_shift, m, counts,
                nullptr, nullptr, 0, d_n,
            d_flags);
        PMH_LAUNCHED("query_kernel<count>");
    }
    return PMH_OK;
}

extern "C" int pmh_lsh_query(pmh_ctx ctx, pmh_index X, const uint32_t* d_qhashes, int64_t Q,
                             int64_t* d_row_ptr, int32_t* d_cand, int64_t cand_capacity,
                             int64_t* h_total, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!X || !d_row_ptr || !h_total || Q < 0 || (Q > 0 && !d_qhashes) || cand_capacity < 0)
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    *h_total = 0;
    if (Q == 0) {
        PMH_CUDA_TRY(cudaMemsetAsync(d_row_ptr, 0, sizeof(int64_t), s));
        return PMH_OK;
    }
    int64_t* counts = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_QUERY, sizeof(int64_t) * (size_t)Q, (void**)&counts));
    // the count pass stages its sorted rows in a pool of up to 4,096 ids per query
    // (at most 64M ids); rows past the pool are joined again by the fill pass
    void* stage = nullptr;
    int64_t pool_ints = 0;
    if (X->params.bands >= 16) {
        pool_ints = std::min<int64_t>(Q * 4096, 64ll << 20);
        PMH_TRY(pmh_scratch(ctx, SCR_JOIN, pmh_join_stage_bytes(Q, pool_ints), &stage));
    }
    PMH_TRY(pmh_launch_query(X, d_qhashes, Q, nullptr, counts, nullptr, nullptr, 0, stage, pool_ints,
                             nullptr, false, s));
    PMH_TRY(pmh_exclusive_scan_i64(ctx, counts, d_row_ptr, Q, s));
    PMH_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, d_row_ptr + Q, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t total = ctx->h_pinned[0];
    *h_total = total;
    if (total > cand_capacity)
        return pmh_set_error(PMH_ERR_CAPACITY, "%lld candidates > capacity %lld", (long long)total,
                             (long long)cand_capacity);
    if (total == 0) return PMH_OK;
    if (!d_cand) return pmh_set_error(PMH_ERR_ARG, "null candidate buffer");
    return pmh_launch_query(X, d_qhashes, Q, nullptr, nullptr, d_row_ptr, d_cand, cand_capacity,
                            stage, pool_ints, nullptr, true, s);
}

extern "C" int pmh_lsh_query_fill(pmh_ctx ctx, pmh_index X, const uint32_t* d_qhashes, int64_t Q,
                                  const int64_t* d_row_ptr, int32_t* d_cand, int64_t cand_capacity,
                                  void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!X || !d_row_ptr || Q < 0 || (Q > 0 && (!d_qhashes || !d_cand)) || cand_capacity < 0)
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    if (Q == 0) return PMH_OK;
    return pmh_launch_query(X, d_qhashes, Q, nullptr, nullptr, d_row_ptr, d_cand, cand_capacity,
                            nullptr, 0, nullptr, true, (cudaStream_t)stream);
}

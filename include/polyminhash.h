/*
 * polyminhash.h -- C ABI of the GB300 (sm_103a) PolyMinHash library.
 *
 * PolyMinHash (arXiv 2511.16576) signs a polygon P with m = K MinHash values:
 * h_k(P) is the index of the first point of hash k's seeded uniform point
 * stream that lands inside P (Definition 2, Algorithm 1).  Two polygons agree
 * on one hash with probability J(P, Q) = area(P n Q) / area(P u Q)
 * (Theorem 1), so signatures bucket similar polygons together (hashmap
 * filtering, Sec. 3.2 after Theorem 1 and Sec. 5.2) and estimate Jaccard.
 *
 * Conventions
 *  - Every call returns PMH_OK (0) or a negative PMH_ERR_* code; the message
 *    of the last failure on the calling thread is pmh_last_error().
 *  - Array arguments named d_* are DEVICE pointers owned by the caller
 *    (for example torch tensors); h_* are host pointers.  Handles
 *    (pmh_ctx, pmh_polys, pmh_index) are owned by the library and released by
 *    their *_destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue their kernels on it and return without waiting,
 *    unless the description says "synchronises".
 *  - There is no CPU fallback: on a machine without a usable sm_103a GPU every
 *    compute call fails with PMH_ERR_CUDA.
 *
 * Geometry and the readings of the paper used by every call
 *  - A polygon is a simple ring of n >= 3 int32 vertices (x, y) given once
 *    (the closing vertex is not repeated); edges are (v_i, v_{(i+1) mod n}).
 *    Coordinates must satisfy |x|, |y| <= 2^20.
 *  - The sampling domain is the integer lattice [0, 65536)^2 (the paper's
 *    global MBR, Sec. 3.1, fixed for all data sets).  Point i of stream k is
 *    v = mix64(s_k + (i+1) * G) with G = 0x9E3779B97F4A7C15,
 *    s_k = mix64(seed + (k+1) * G) and mix64 the SplitMix64 output function;
 *    x = v & 0xFFFF, y = (v >> 16) & 0xFFFF.
 *  - A lattice point p is inside P iff p + (e1, e2), 0 < e2 << e1
 *    infinitesimal, lies inside P (even-odd rule); this makes membership
 *    exact, monotone under containment and additive over tilings.
 *  - h_k(P) = min{ i in [0, T) : point i of stream k is inside P }, else T
 *    (0-based count of rejected attempts, capped at T <= 2^31).
 */
#ifndef POLYMINHASH_H
#define POLYMINHASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMH_OK 0
#define PMH_ERR_ARG (-1)      /* invalid argument (null, size, shape) */
#define PMH_ERR_RANGE (-2)    /* input data out of the supported range */
#define PMH_ERR_CAPACITY (-3) /* an output buffer is too small */
#define PMH_ERR_CUDA (-4)     /* a CUDA runtime call or kernel failed */
#define PMH_ERR_TIMEOUT (-5)  /* a bounded device-side wait gave up */
#define PMH_ERR_STATE (-6)    /* handle used in the wrong state */
#define PMH_ERR_NOMEM (-7)    /* device or host allocation failed */

#define PMH_INVALID_KEY 0xFFFFFFFFFFFFFFFFull

typedef struct pmh_ctx_s* pmh_ctx;
typedef struct pmh_polys_s* pmh_polys;
typedef struct pmh_index_s* pmh_index;
typedef struct pmh_rerank_s* pmh_rerank;

/* Signature and banding parameters.
 *   seed      global stream seed (Sec. 3.2: fixed seeds per hash function)
 *   K         signature length m (Definition 2), 1 <= K <= 4096
 *   T         stream cap, 1 <= T <= 2^31; a hash that never hits is T
 *   bands     number of LSH bands b, rows = K / bands (K % bands == 0),
 *             1 <= bands <= 128
 *   rows      r, must equal K / bands
 *   lsh_seed  seed of the band-key fingerprint
 *   flags     0 or PMH_FLAG_STREAM_INDEX | PMH_FLAG_COVERAGE_MASK */
/* pmh_params.flags: sign through the stream index (same hashes, much less
 * work for small polygons).  The first call with a given (seed, K) builds the
 * index of the first 65,536 / 32,768 / 8,192 / 1,048,576 points of each stream,
 * bucketed by cell of a 128 x 128 / 64 x 64 / 32 x 32 / 512 x 512 grid (8 bytes
 * per point and per (cell, hash) record: about K * 11.5 MB of device memory,
 * kept by the context; that call synchronises); later calls reuse it.
 * Each polygon's form (index or walk) and grid level are planned at upload from
 * its box and area. */
#define PMH_FLAG_STREAM_INDEX 1u
/* pmh_params.flags: decide bounding-box candidates of the walk through a
 * precomputed per-polygon 16 x 16 coverage mask where it can (cells no edge
 * touches are wholly inside or outside), running the exact edge test only in
 * boundary cells.  Same hashes.  The masks are built on the first such call for
 * a polygon set (64 bytes per polygon of up to 256 vertices) and kept with it.
 * Without this flag the signing kernels for polygons of up to 256 vertices
 * build a 32 x 32 mask in shared memory themselves; with it, those polygons that
 * take the walk form use the precomputed mask instead. */
#define PMH_FLAG_COVERAGE_MASK 2u

typedef struct {
    uint64_t seed;
    uint32_t K;
    uint32_t T;
    uint32_t bands;
    uint32_t rows;
    uint64_t lsh_seed;
    uint32_t flags;
    uint32_t reserved;
} pmh_params;

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char* pmh_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int pmh_version(void);

/* Create a context on CUDA device `device`: it owns scratch buffers and a
 * device status word.  Not thread-safe: use one context per host thread.
 * Errors: PMH_ERR_ARG (null out), PMH_ERR_CUDA (no such device / not sm_103). */
int pmh_create(pmh_ctx* out, int device);
/* Release a context.  Handles made with it (polygons, indexes, graphs) stay
 * releasable afterwards but may no longer be used in compute calls. */
int pmh_destroy(pmh_ctx ctx);

/* A0 -- upload polygons (Sec. 3.1 preprocessing: local MBRs).
 * Copies n_polys polygons into library-owned device memory and computes each
 * polygon's half-open bounding box clipped to the domain, twice its signed
 * area (exact int64 shoelace), its signing plan (indexed or walk form, grid
 * level) and the order in which the signing kernels take the polygons.
 *   d_xy       int32 [n_vertices][2], interleaved (x, y), device
 *   d_offsets  int64 [n_polys + 1], offsets[0] = 0, offsets[n_polys] =
 *              n_vertices, polygon p = vertices offsets[p] .. offsets[p+1]-1
 * Synchronises `stream` once to report validation failures.
 * Errors: PMH_ERR_ARG (null, n_polys < 0, n_polys >= 2^31),
 *         PMH_ERR_RANGE (offsets not increasing, a polygon with < 3 vertices,
 *         a coordinate beyond 2^20), PMH_ERR_NOMEM, PMH_ERR_CUDA. */
int pmh_poly_upload(pmh_ctx ctx, const int32_t* d_xy, const int64_t* d_offsets,
                    int64_t n_polys, int64_t n_vertices, pmh_polys* out, void* stream);

/* Same as pmh_poly_upload with HOST arrays (pageable or pinned); the
 * host-to-device copies run on `stream` inside the call. */
int pmh_poly_upload_host(pmh_ctx ctx, const int32_t* h_xy, const int64_t* h_offsets,
                         int64_t n_polys, int64_t n_vertices, pmh_polys* out, void* stream);

/* Upload new polygons into an existing set with the same n_polys and
 * n_vertices (HOST arrays if host_memory != 0, else device), keeping the
 * set's vertex, offset, box and area buffers -- so a query graph that
 * refines against the set stays valid -- and rebuilding everything else as
 * pmh_poly_upload does.  Synchronises `stream` before and after; work on other
 * streams that reads the set meanwhile races.  Errors: as pmh_poly_upload,
 * and PMH_ERR_ARG if the sizes differ from the set's; on a validation error
 * the set holds the rejected data and must not be signed. */
int pmh_poly_reload(pmh_polys polys, const int32_t* xy, const int64_t* offsets, int64_t n_polys,
                    int64_t n_vertices, int host_memory, void* stream);

/* Number of polygons and vertices of an uploaded set. */
int pmh_polys_info(pmh_polys polys, int64_t* n_polys, int64_t* n_vertices);

/* Copy the per-polygon preprocessing out (for inspection):
 *   d_bbox   int32 [n_polys][4] = x0, y0, x1, y1: lattice points inside P
 *            satisfy x0 <= x < x1, y0 <= y < y1 (already clipped to the domain)
 *   d_area2  int64 [n_polys] twice the signed area
 * Either pointer may be NULL. */
int pmh_polys_prep(pmh_polys polys, int32_t* d_bbox, int64_t* d_area2, void* stream);
int pmh_polys_destroy(pmh_polys polys);

/* A1 -- MinHash signatures (Definition 2, Algorithm 1; 0-based, cap T).
 *   d_hashes  uint32 [n_polys][K] row-major, written completely.
 * Hashes are exact: bit-identical to the definition above.  The first call on
 * a context with PMH_FLAG_STREAM_INDEX builds the stream index for (seed, K),
 * and the first call on a polygon set without it builds the set's cost order;
 * both synchronise the stream once.  Calls on one polygon set from several
 * host threads at once must be serialised by the caller.
 * Errors: PMH_ERR_ARG (null, bad K/T), PMH_ERR_CUDA. */
int pmh_minhash_sign(pmh_ctx ctx, pmh_polys polys, const pmh_params* params,
                     uint32_t* d_hashes, void* stream);

/* Build (or reuse) the context's stream index for params->seed and K ahead of
 * the first indexed pmh_minhash_sign call.  Synchronises. */
int pmh_stream_index_build(pmh_ctx ctx, const pmh_params* params, void* stream);

/* Algorithmic work of the last pmh_minhash_sign call on this context
 * (synchronises): h_counts[0] stream points examined by walks (up to each
 * result), [1] grid cells read by the indexed form, [2] stream-index entries
 * read, [3] bounding-box candidates ordered, [4] polygon edges tested,
 * [5] candidates decided by a polygon's coverage mask without edge tests
 * (h_counts holds 6 values). */
int pmh_sign_work(pmh_ctx ctx, uint64_t* h_counts);

/* Whether later signing calls on this context record those counts (1, the
 * default) or run kernels built without the counters (0; pmh_sign_work and
 * pmh_sign_report then return zeros for them).  The counters are measurement
 * support only: the hashes are the same either way. */
int pmh_sign_count_work(pmh_ctx ctx, int enable);

/* Measurement support (no counterpart in the paper).  With the stream index,
 * pmh_minhash_sign signs every polygon in one persistent launch (the unified
 * kernel: indexed or walk form per polygon); without it, or with
 * PMH_FLAG_COVERAGE_MASK, it runs the walk kernel over every polygon.
 * pmh_sign_timing(ctx, 1) makes later signing calls on this context record
 * CUDA events around each of the two on the caller's stream, without
 * synchronising (0 stops it; at most 1024 calls are kept).
 * pmh_sign_report (synchronises) returns h_ms[0] / h_ms[1] = mean
 * milliseconds of the unified / walk kernel over the calls recorded since
 * the previous report (0 for a kernel the calls did not run), h_ms[2] =
 * their number (h_ms holds 3 floats; NULL: skip; the recorded calls are then
 * forgotten), and h_counts[0..5] / [6..11] = the six work counts of
 * pmh_sign_work for each kernel alone in the last signing call (NULL: skip).
 * Errors: PMH_ERR_ARG (null context), PMH_ERR_CUDA. */
int pmh_sign_timing(pmh_ctx ctx, int enable);
int pmh_sign_report(pmh_ctx ctx, float* h_ms, uint64_t* h_counts);

/* A2 -- band keys (hashmap keys of Sec. 3.2 after Theorem 1, one per band).
 * Band j covers hashes j*r .. j*r+r-1; a = mix64(lsh_seed + (j+1)*G), then
 * a = mix64(a ^ h) for each of its r hashes; a band holding T has key
 * PMH_INVALID_KEY, a valid key equal to it is replaced by it minus one.
 *   d_hashes uint32 [n][K]; d_keys uint64 [n][bands]. */
int pmh_band_keys(pmh_ctx ctx, const uint32_t* d_hashes, int64_t n, const pmh_params* params,
                  uint64_t* d_keys, void* stream);

/* A3 -- build the bucket index of n database signatures (one hashmap per
 * band): band keys plus a stable radix sort of (band, key) with ids.  The
 * index keeps its own copy of the hashes it needs, so d_hashes may be freed
 * afterwards.  Errors: PMH_ERR_ARG, PMH_ERR_NOMEM, PMH_ERR_CUDA. */
int pmh_lsh_build(pmh_ctx ctx, const uint32_t* d_hashes, int64_t n, const pmh_params* params,
                  pmh_index* out, void* stream);
/* Rebuild an index in place from n new signatures (n and the parameters of the
 * index unchanged): the index keeps its buffers, so a query graph captured on
 * it stays valid.  Enqueued on `stream`; a query on another stream that reads
 * the index meanwhile races.  Errors: PMH_ERR_ARG (other context or size),
 * PMH_ERR_CUDA. */
int pmh_lsh_rebuild(pmh_ctx ctx, pmh_index index, const uint32_t* d_hashes, int64_t n,
                    void* stream);
int pmh_index_destroy(pmh_index index);

/* A4 -- bucket join.  Candidates of query q: every database id p with some
 * band j whose r-tuple is valid (no T) in both and equal in both, ascending,
 * without duplicates, as CSR:
 *   d_row_ptr int64 [Q + 1] (device), d_cand int32 [cand_capacity] (device)
 *   h_total   (host) receives the number of candidates over all queries.
 * Synchronises `stream` once (to learn the total).  With cand_capacity <
 * total, d_cand is left unwritten, d_row_ptr is still written, and the call
 * returns PMH_ERR_CAPACITY: call again with a larger buffer.  From 16 bands the
 * counting pass keeps its sorted rows in context scratch (8 bytes per query and
 * up to 4,096 ids per query, at most 64M ids) and the filling pass copies them;
 * rows past that pool are joined again.  Errors also: PMH_ERR_NOMEM (scratch). */
int pmh_lsh_query(pmh_ctx ctx, pmh_index index, const uint32_t* d_qhashes, int64_t Q,
                  int64_t* d_row_ptr, int32_t* d_cand, int64_t cand_capacity, int64_t* h_total,
                  void* stream);

/* Second half of pmh_lsh_query for callers that sized the candidate buffer
 * from a first call (cand_capacity = 0 gives the total and writes d_row_ptr):
 * fills d_cand from that d_row_ptr without recounting.  cand_capacity must be
 * at least the total (else nothing is written).  Does not synchronise. */
int pmh_lsh_query_fill(pmh_ctx ctx, pmh_index index, const uint32_t* d_qhashes, int64_t Q,
                       const int64_t* d_row_ptr, int32_t* d_cand, int64_t cand_capacity,
                       void* stream);

/* A5 -- agreement estimate (Theorem 1: Pr[h_k(q) = h_k(p)] = J(q, p)).
 * For every CSR pair (q, d_cand[e]): d_count[e] = #{k : h_k(q) = h_k(p) != T}
 * (J estimate = count / K) and, if d_bandmask is not NULL, bit j of
 * d_bandmask[e] set iff band j (j < 32) is valid and equal in both.
 *   d_qhashes uint32 [Q][K], d_dbhashes uint32 [N][K], d_row_ptr int64 [Q+1],
 *   d_cand int32 [row_ptr[Q]] (ids < N; not checked). */
int pmh_jaccard_estimate(pmh_ctx ctx, const uint32_t* d_qhashes, const uint32_t* d_dbhashes,
                         const int64_t* d_row_ptr, const int32_t* d_cand, int64_t Q,
                         const pmh_params* params, uint16_t* d_count, uint32_t* d_bandmask,
                         void* stream);

/* A6 -- top-m of every candidate row.  Order: (count desc, id asc), or with
 * d_score != NULL (float per pair, e.g. a learned Jaccard) (score desc, id
 * asc).  d_out_ids int32 [Q][m] (-1 padded), d_out_n int32 [Q]. 1 <= m <= 1024.
 * Counts are agreement counts (at most K <= 4,096); a larger count ranks as
 * 4,096.  Does not synchronise. */
int pmh_topm(pmh_ctx ctx, const int64_t* d_row_ptr, const int32_t* d_cand,
             const uint16_t* d_count, const float* d_score, int64_t Q, int32_t m,
             int32_t* d_out_ids, int32_t* d_out_n, void* stream);

/* Fixed-width lists (d_ids [Q][m] as written by pmh_topm, d_n [Q] kept per
 * row) to compact CSR: d_row_ptr int64 [Q + 1], d_cand int32 (capacity Q*m).
 * Used to rerank a count-ordered shortlist with the learned scores. */
int pmh_lists_to_csr(pmh_ctx ctx, const int32_t* d_ids, const int32_t* d_n, int64_t Q, int32_t m,
                     int64_t* d_row_ptr, int32_t* d_cand, void* stream);

/* A8 -- exact refinement (Sec. 5.2 refinement phase): for every query q and
 * each of its d_n[q] listed ids (d_ids [Q][m]), the exact Jaccard
 * J = area(q n p) / area(q u p) in fp64; keeps the best k by (J desc, id asc).
 *   d_top_ids int32 [Q][k] (-1 padded), d_top_j double [Q][k].
 * 1 <= k <= m <= 1024. */
int pmh_refine_topk(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_ids,
                    const int32_t* d_n, int64_t Q, int32_t m, int32_t k, int32_t* d_top_ids,
                    double* d_top_j, void* stream);

/* Exact Jaccard of explicit pairs (d_qid[e], d_pid[e]) -> d_j[e] (fp64). */
int pmh_pair_jaccard(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const int32_t* d_qid,
                     const int32_t* d_pid, int64_t n_pairs, double* d_j, void* stream);

/* A9 -- batching: signing-kernel variants and their autotuner.
 * The signing kernel exists in PMH_SIGN_VARIANTS shapes (points per lane per
 * round x warps per block).  pmh_sign_autotune times every variant on the
 * polygons of `sample` (typically a few thousand polygons of the workload),
 * stores the fastest in the context (later pmh_minhash_sign calls use it) and
 * returns its index; h_ms (optional, PMH_SIGN_VARIANTS floats) receives each
 * variant's time.  Synchronises.  pmh_sign_set_variant(ctx, -1) restores the
 * default.  Hashes do not depend on the variant. */
#define PMH_SIGN_VARIANTS 6
int pmh_sign_autotune(pmh_ctx ctx, pmh_polys sample, const pmh_params* params, int* h_best,
                      float* h_ms);
int pmh_sign_set_variant(pmh_ctx ctx, int variant);
int pmh_sign_variant_info(int variant, int* points_per_lane, int* warps_per_block);

/* A9 -- batching: the query pipeline as one CUDA graph.
 * pmh_qgraph_create captures, on buffers the graph owns, the chain
 * A0 prep -> y-slab lists of the polygons above 256 vertices -> A1 sign (one
 * launch of the unified kernel: through the stream index when the index's
 * params carry PMH_FLAG_STREAM_INDEX, which this call builds if needed and
 * which must not be rebuilt for other parameters while the graph lives) ->
 * A4 join -> A5 agreement -> A6 top-m per query -> (k > 0) A8 exact
 * refinement of the top-m lists to the top-k by (J desc, id asc) against the
 * polygon set cfg->db, for batches of at most max_queries polygons holding at
 * most max_vertices vertices.  With cfg->rerank (A7, learned form) the top-m
 * are the m best by the reranker's predicted Jaccard among the `shortlist`
 * best by agreement count (m <= shortlist <= 1024, K a multiple of 32, db the
 * polygon set `index` was built from); the reranker's weights are read at
 * every replay, so later training is seen.  `index`, db and the reranker must
 * outlive the graph.  The slab lists get fixed buffers (a table entry per
 * slab, four list entries per vertex); a polygon whose lists do not fit is
 * tested over all its edges.  Synchronises; 0 <= k <= m <= 1024.
 * pmh_qgraph_run copies one batch (xy int32 [n_vertices][2], offsets int64
 * [n_queries + 1], HOST arrays if host_memory != 0, else device) into the
 * graph's inputs and replays the graph on `stream`: it neither allocates nor
 * synchronises.  Batches beyond the graph's sizes fail with PMH_ERR_RANGE; a
 * stream index rebuilt since the capture fails with PMH_ERR_STATE.
 * pmh_qgraph_outputs returns device pointers (owned by the graph, valid until
 * pmh_qgraph_destroy, rewritten by every run): hashes uint32 [max_queries][K],
 * row_ptr int64 [max_queries + 1], cand int32 [cand_capacity], count uint16
 * [cand_capacity], top_ids int32 [max_queries][m] (-1 padded), top_n int32
 * [max_queries]; rows past the batch are empty.  pmh_qgraph_refined returns
 * the refined top-k (int32 ids [max_queries][k], -1 padded; fp64 J, -1 in
 * empty slots; rows past the batch are not written), PMH_ERR_STATE if k == 0.
 * pmh_qgraph_status synchronises `stream` and reports the last run's status
 * bits (1, 2, 4: invalid polygons -- offsets, fewer than 3 vertices,
 * coordinate range -- nothing computed; 8: more candidates than
 * cand_capacity, rows not written, agreement, top-m and refinement skipped;
 * 16: a bounded wait on the tensor cores in the reranker's forward pass ran
 * out, scores not written) and its candidate total. */
typedef struct pmh_qgraph_s* pmh_qgraph;
typedef struct {
    int64_t max_queries, max_vertices, cand_capacity;
    int32_t m;           /* candidates per query kept for refinement (top-m) */
    int32_t k;           /* refined top-k (0: no refinement) */
    pmh_polys db;        /* the indexed polygon set (refinement, learned features) */
    pmh_rerank rerank;   /* learned form (NULL: rank by agreement count) */
    int32_t shortlist;   /* learned form: candidates by count rescored per query */
    int32_t options;     /* bit 0: learned form in one fused launch (PMH_QGRAPH_FUSED_SELECT) */
} pmh_qgraph_config;
/* options bit 0 (learned form, shortlist dividing 128, K a multiple of 32 up to
 * 4,096): features, scores and the top-m by score in one launch instead of four
 * (feature rows, forward pass, top-m, with the lists compacted first); the same
 * lists either way.  Off by default: on the 10M combined workload the separate
 * launches are the faster form. */
#define PMH_QGRAPH_FUSED_SELECT 1
int pmh_qgraph_create(pmh_ctx ctx, pmh_index index, const pmh_qgraph_config* cfg,
                      pmh_qgraph* out);
int pmh_qgraph_run(pmh_qgraph graph, const int32_t* xy, const int64_t* offsets, int64_t n_queries,
                   int64_t n_vertices, int host_memory, void* stream);
int pmh_qgraph_outputs(pmh_qgraph graph, uint32_t** d_hashes, int64_t** d_row_ptr,
                       int32_t** d_cand, uint16_t** d_count, int32_t** d_top_ids,
                       int32_t** d_top_n);
int pmh_qgraph_refined(pmh_qgraph graph, int32_t** d_top_ids, double** d_top_j);
int pmh_qgraph_status(pmh_qgraph graph, int* h_flags, int64_t* h_total, void* stream);
int pmh_qgraph_destroy(pmh_qgraph graph);

/* A7 -- learned reranker (not in the paper): an MLP 40 -> 64 -> 64 -> 1
 * (ReLU, ReLU, sigmoid) predicting the Jaccard similarity of a (query,
 * candidate) pair, trained on the GPU by mean squared error against exact
 * Jaccard.  bf16 weights and activations on the tensor cores, fp32
 * accumulation and fp32 master weights (Adam): the forward pass (scoring) as
 * tcgen05 MMAs from shared memory into tensor-memory accumulators, training
 * with mma.sync.
 * Packed parameter layout (PMH_RERANK_PARAMS floats): w1 [64][40] (out, in),
 * b1 [64], w2 [64][64], b2 [64], w3 [64], b3 [1].
 * Features (pmh_rerank_features): bf16 [E][48] per CSR pair, columns
 *   0..31 group-match bits (group j = hashes j*K/32 .. (j+1)*K/32-1 all equal
 *          and not T), 32 agreement count / K, 33-34 log2(area) / 32 of query
 *          and candidate, 35-36 log2(vertex count) / 16, 37 / 38 the number
 *          of hashes with h_k(query) < h_k(candidate) / h_k(query) >
 *          h_k(candidate), over K, 39 the upper bound m / (|q| + |p| - m) of
 *          J with m = min(|q|, |p|, overlap area of the two bounding boxes),
 *          40..47 zero.  By the min form of the hash (Theorem 1's proof),
 *          h_k(q) < h_k(p) happens with probability area(q \ p) / area(q u p)
 *          and h_k(q) > h_k(p) with area(p \ q) / area(q u p): with the exact
 *          areas, the two counts sharpen the estimate of the overlap where the
 *          areas differ; the bound is a geometric prior the hashes lack.
 *   K must be a multiple of 32.
 * pmh_rerank_forward writes a score in (0, 1) per feature row (feed it to
 * pmh_topm as d_score); d_feat must be 16-byte aligned; it synchronises
 * `stream` and returns PMH_ERR_CUDA if a bounded wait on the tensor cores ran
 * out (scores not written).  pmh_rerank_gradients computes the loss (mean over
 * n_rows) and the packed gradients of one batch into the reranker (and
 * copies them to d_grads / d_loss when not NULL); pmh_rerank_adam_step
 * applies them.  set/get move the packed fp32 master weights (synchronise). */
#define PMH_RERANK_IN 40
#define PMH_RERANK_HIDDEN 64
#define PMH_RERANK_PARAMS 6849
int pmh_rerank_create(pmh_ctx ctx, pmh_rerank* out);
int pmh_rerank_destroy(pmh_rerank r);
int pmh_rerank_set_weights(pmh_rerank r, const float* h_params);
int pmh_rerank_get_weights(pmh_rerank r, float* h_params);
int pmh_rerank_features(pmh_ctx ctx, pmh_polys queries, pmh_polys db, const uint32_t* d_qhashes,
                        const uint32_t* d_dbhashes, const int64_t* d_row_ptr,
                        const int32_t* d_cand, int64_t Q, const pmh_params* params,
                        uint16_t* d_feat, void* stream);
int pmh_rerank_forward(pmh_rerank r, const uint16_t* d_feat, int64_t n_rows, float* d_score,
                       void* stream);
int pmh_rerank_gradients(pmh_rerank r, const uint16_t* d_feat, const float* d_label,
                         int64_t n_rows, float* d_grads, float* d_loss, void* stream);
int pmh_rerank_adam_step(pmh_rerank r, float lr, float beta1, float beta2, float eps,
                         void* stream);

/* Allocation-free signing (the paper has no counterpart: this is a deployment
 * entry point).  Same hashes as pmh_minhash_sign, for callers that must not
 * let a library allocate device memory: processes that reserve their whole
 * device-memory budget up front, hosts whose memory is owned by a caching
 * allocator that a side cudaMalloc would fragment or starve, and
 * latency-critical loops that cannot absorb the device-wide synchronisation of
 * cudaFree.  It takes raw device arrays instead of a pmh_polys handle and needs
 * no pmh_ctx:
 *   d_xy       int32 [n_vertices][2] interleaved (x, y), device
 *   d_offsets  int64 [n_polys + 1], device (same layout as pmh_poly_upload)
 *   d_hashes   uint32 [n_polys][K], device, written completely
 * It runs on the current device and calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch (work-queue ticket, validation
 * word, one bounding box per polygon) is a fixed device array of
 * PMH_NOALLOC_MAX_POLYS + 1 16-byte entries (4 MiB) that every GPU loading
 * the library holds until the process exits; n_polys above
 * PMH_NOALLOC_MAX_POLYS is rejected with PMH_ERR_RANGE before any GPU work.
 * d_xy, d_offsets and d_hashes must be device (or managed) memory of the
 * current device; host pointers and other GPUs' memory are refused with
 * PMH_ERR_ARG before anything is launched.
 * The first call on a device looks up the array's device address, once per
 * device, and keeps it for the life of the process: after a
 * cudaDeviceReset of that device the kept address is stale, so do not use
 * this entry point across a device reset.  Every call shares the one array
 * and clears its ticket and flags itself, so calls that overlap on the GPU
 * (two streams, two threads) race: serialise them.  Every call synchronises
 * `stream` once to read the validation word (the same error codes as
 * pmh_poly_upload), so the entry point cannot be called while `stream` is
 * being captured into a CUDA graph. */
#define PMH_NOALLOC_MAX_POLYS 262144
int pmh_minhash_sign_noalloc(const int32_t* d_xy, const int64_t* d_offsets, int64_t n_polys,
                             int64_t n_vertices, const pmh_params* params, uint32_t* d_hashes,
                             void* stream);

/* Brute-force candidates (the exact search the paper compares against,
 * Sec. 5.2): CSR of every database polygon whose bounding box overlaps the
 * query's with positive area (the only polygons with J > 0), ids ascending.
 * Same two-pass capacity protocol and synchronisation as pmh_lsh_query. */
int pmh_bbox_join(pmh_ctx ctx, pmh_polys queries, pmh_polys db, int64_t* d_row_ptr,
                  int32_t* d_cand, int64_t cand_capacity, int64_t* h_total, void* stream);

/* Integer-ALU throughput probe used as the roofline denominator: runs a
 * fixed mix of 32-bit integer instructions (add, logic, shift, multiply-add)
 * on every SM and reports integer instructions per second (thread level).
 * Synchronises. */
int pmh_probe_int_peak(pmh_ctx ctx, double* h_int_ops_per_s, double* h_seconds);

/* Number of kernels this library has launched in this process (all
 * contexts); used to count launches inside a timed region. */
int64_t pmh_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif

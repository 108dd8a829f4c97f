// graph.cu -- A9: the query pipeline captured once as a CUDA graph.
//
// For query batches of up to max_queries polygons (at most max_vertices
// vertices in all), the steps prep (A0), y-slab edge lists of the polygons
// above the staged size, sign (A1: one launch of the unified kernel, through
// the stream index when the index's parameters ask for it), bucket join (A4,
// count + scan + fill), agreement (A5), top-m (A6) and, with a database
// polygon set, exact refinement of the top-m to the top-k (A8) are captured on
// fixed, graph-owned buffers; with a reranker the top-m are chosen by its
// predicted Jaccard among a shortlist by agreement count (A7, learned form).
// A replay copies the batch into the input buffers, writes the batch size into
// a device word and launches the graph:
// no host synchronisation, no allocation.  Data-dependent sizes stay on the
// device: kernels read the batch size from the device word, the slab lists of
// a polygon that does not fit the fixed buffers are left out (that polygon is
// tested over all its edges), the join writes its rows only if the candidate
// total fits the capacity, and a device status word records failures (bits
// 0-2 invalid polygons, bit 3 candidate overflow) which make the later stages
// do nothing; pmh_qgraph_status reads it.
#include <algorithm>

#include "pmh_internal.cuh"

struct pmh_qgraph_s {
    pmh_ctx ctx = nullptr;
    int device = 0;
    pmh_index index = nullptr;
    pmh_polys db = nullptr;           // refinement target (nullptr: no refinement)
    pmh_params P{};
    int64_t maxQ = 0, maxV = 0, cap = 0;
    int m = 0, k = 0;
    int2* xy = nullptr;
    int64_t* off = nullptr;
    int4* bbox = nullptr;
    int64_t* area2 = nullptr;
    uint32_t* hashes = nullptr;
    SlabInfo* slab_info = nullptr;    // y-slab lists of the batch's large polygons
    int64_t* slab_sizes = nullptr;
    int64_t* slab_sums = nullptr;
    int32_t* slab_ptr = nullptr;
    int32_t* slab_cursor = nullptr;
    int32_t* slab_edges = nullptr;
    int64_t cap_ptr = 0, cap_edges = 0;
    int64_t* counts = nullptr;
    void* join_stage = nullptr;       // join rows sorted by the count pass (nullable): a pool of cap ids
    int64_t* row_ptr = nullptr;
    int32_t* cand = nullptr;
    uint16_t* count16 = nullptr;
    int32_t* top_ids = nullptr;
    int32_t* top_n = nullptr;
    // learned form: shortlist by count -> compact lists -> features -> scores
    pmh_rerank rerank = nullptr;
    int shortlist = 0;
    bool fused_select = false;  // features, scores and top-m in one launch
    int32_t* sl_ids = nullptr;
    int32_t* sl_n = nullptr;
    int64_t* sl_counts = nullptr;
    int64_t* sl_sums = nullptr;
    int64_t* sl_row_ptr = nullptr;
    int32_t* sl_cand = nullptr;
    float2* qfeat = nullptr;
    uint16_t* feat = nullptr;
    float* score = nullptr;
    double* jv = nullptr;             // exact J of the top-m lists
    int32_t* ref_ids = nullptr;       // refined top-k
    double* ref_j = nullptr;
    int* flags = nullptr;
    int64_t* d_n = nullptr;
    unsigned long long* ticket = nullptr;  // [2]: signing grid, refinement grid
    int64_t* scan_sums = nullptr;
    const uint2* sidx_cell = nullptr;  // the stream index the graph captured (nullptr: none)
    int64_t kernels = 0;               // kernel launches per replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

__global__ void set_batch_kernel(int64_t* d_n, int64_t n) { *d_n = n; }

}  // namespace

extern "C" int pmh_qgraph_destroy(pmh_qgraph g)
{
    if (!g) return PMH_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    void* bufs[] = {g->xy,        g->off,        g->bbox,       g->area2,     g->hashes,
                    g->slab_info, g->slab_sizes, g->slab_sums,  g->slab_ptr,  g->slab_cursor,
                    g->slab_edges, g->counts,    g->row_ptr,    g->cand,      g->count16,
                    g->top_ids,   g->top_n,      g->jv,         g->ref_ids,   g->ref_j,
                    g->flags,     g->d_n,        g->ticket,     g->scan_sums, g->sl_ids,
                    g->sl_n,      g->sl_counts,  g->sl_sums,    g->sl_row_ptr, g->sl_cand,
                    g->qfeat,     g->feat,       g->score,     g->join_stage};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete g;
    return PMH_OK;
}

extern "C" int pmh_qgraph_create(pmh_ctx ctx, pmh_index index, const pmh_qgraph_config* cfg,
                                 pmh_qgraph* out)
{
    if (!out) return pmh_set_error(PMH_ERR_ARG, "null out");
    *out = nullptr;
    PMH_TRY(pmh_check_device(ctx));
    if (!cfg) return pmh_set_error(PMH_ERR_ARG, "null config");
    const int64_t max_queries = cfg->max_queries, max_vertices = cfg->max_vertices;
    const int64_t cand_capacity = cfg->cand_capacity;
    const int32_t m = cfg->m, k = cfg->k, S = cfg->rerank ? cfg->shortlist : 0;
    pmh_polys db = cfg->db;
    if (!index || max_queries < 1 || max_queries >= (1ll << 31) || max_vertices < 3 ||
        cand_capacity < 1 || m < 1 || m > 1024 || k < 0 || k > m || ((k > 0 || cfg->rerank) && !db))
        return pmh_set_error(PMH_ERR_ARG, "bad graph sizes (0 <= k <= m <= 1024; refinement and the "
                                          "learned form need db)");
    if (cfg->rerank && (S < m || S > 1024 || index->params.K % 32 != 0 || db->n != index->n))
        return pmh_set_error(PMH_ERR_ARG, "learned form: m <= shortlist <= 1024, K a multiple of 32, "
                                          "db the indexed set");
    if (cfg->options & ~PMH_QGRAPH_FUSED_SELECT) return pmh_set_error(PMH_ERR_ARG, "unknown graph options");
    if (cfg->rerank && (cfg->options & PMH_QGRAPH_FUSED_SELECT) &&
        !pmh_rerank_select_fits(S, (int)index->params.K))
        return pmh_set_error(PMH_ERR_ARG, "fused selection: the shortlist must divide 128 (at least 4), K a "
                                          "multiple of 32 up to 4,096");
    pmh_qgraph g = new pmh_qgraph_s();
    g->ctx = ctx;
    g->device = ctx->device;
    g->index = index;
    g->db = db;
    g->rerank = cfg->rerank;
    g->shortlist = S;
    g->fused_select = cfg->rerank && (cfg->options & PMH_QGRAPH_FUSED_SELECT);
    g->P = index->params;
    g->maxQ = max_queries;
    g->maxV = max_vertices;
    g->cap = cand_capacity;
    g->m = m;
    g->k = k;
    const int64_t Q = max_queries, K = g->P.K;
    // every large polygon has at most n / 4 slabs: the slab tables fit exactly; the
    // edge lists get four entries per vertex (a polygon needing more is left out)
    g->cap_ptr = max_vertices / 4 + Q + 1;
    g->cap_edges = 4 * max_vertices;
    // the stream index is built (or found) now: building it synchronises
    StreamIndexView sidx{};
    if (g->P.flags & PMH_FLAG_STREAM_INDEX) {
        const int rc = pmh_stream_index_get(ctx, &g->P, nullptr, &sidx);
        if (rc != PMH_OK) {
            delete g;
            return rc;
        }
        if (!sidx.ranked) sidx = StreamIndexView{};  // saturated lists: sign by walking
        g->sidx_cell = sidx.cell;
    }
    bool ok = cudaMalloc(&g->xy, sizeof(int2) * max_vertices) == cudaSuccess &&
              cudaMalloc(&g->off, sizeof(int64_t) * (Q + 1)) == cudaSuccess &&
              cudaMalloc(&g->bbox, sizeof(int4) * Q) == cudaSuccess &&
              cudaMalloc(&g->area2, sizeof(int64_t) * Q) == cudaSuccess &&
              cudaMalloc(&g->hashes, sizeof(uint32_t) * Q * K) == cudaSuccess &&
              cudaMalloc(&g->slab_info, sizeof(SlabInfo) * Q) == cudaSuccess &&
              cudaMalloc(&g->slab_sizes, sizeof(int64_t) * 2 * (Q + 1)) == cudaSuccess &&
              cudaMalloc(&g->slab_sums, sizeof(int64_t) * 2 * pmh_scan_sums_size(Q)) == cudaSuccess &&
              cudaMalloc(&g->slab_ptr, sizeof(int32_t) * g->cap_ptr) == cudaSuccess &&
              cudaMalloc(&g->slab_cursor, sizeof(int32_t) * g->cap_ptr) == cudaSuccess &&
              cudaMalloc(&g->slab_edges, sizeof(int32_t) * g->cap_edges) == cudaSuccess &&
              cudaMalloc(&g->counts, sizeof(int64_t) * Q) == cudaSuccess &&
              (index->params.bands < 16 ||
               cudaMalloc(&g->join_stage, pmh_join_stage_bytes(Q, g->cap)) == cudaSuccess) &&
              cudaMalloc(&g->row_ptr, sizeof(int64_t) * (Q + 1)) == cudaSuccess &&
              cudaMalloc(&g->cand, sizeof(int32_t) * cand_capacity) == cudaSuccess &&
              cudaMalloc(&g->count16, sizeof(uint16_t) * cand_capacity) == cudaSuccess &&
              cudaMalloc(&g->top_ids, sizeof(int32_t) * Q * m) == cudaSuccess &&
              cudaMalloc(&g->top_n, sizeof(int32_t) * Q) == cudaSuccess &&
              (S == 0 || (cudaMalloc(&g->sl_ids, sizeof(int32_t) * Q * S) == cudaSuccess &&
                          cudaMalloc(&g->sl_n, sizeof(int32_t) * Q) == cudaSuccess &&
                          cudaMalloc(&g->sl_counts, sizeof(int64_t) * Q) == cudaSuccess &&
                          cudaMalloc(&g->sl_sums, sizeof(int64_t) * pmh_scan_sums_size(Q)) == cudaSuccess &&
                          cudaMalloc(&g->sl_row_ptr, sizeof(int64_t) * (Q + 1)) == cudaSuccess &&
                          cudaMalloc(&g->sl_cand, sizeof(int32_t) * Q * S) == cudaSuccess &&
                          cudaMalloc(&g->qfeat, sizeof(float2) * Q) == cudaSuccess &&
                          cudaMalloc(&g->feat, sizeof(uint16_t) * 48 * Q * S) == cudaSuccess &&
                          cudaMalloc(&g->score, sizeof(float) * Q * S) == cudaSuccess)) &&
              (k == 0 || (cudaMalloc(&g->jv, sizeof(double) * Q * m) == cudaSuccess &&
                          cudaMalloc(&g->ref_ids, sizeof(int32_t) * Q * k) == cudaSuccess &&
                          cudaMalloc(&g->ref_j, sizeof(double) * Q * k) == cudaSuccess)) &&
              cudaMalloc(&g->flags, sizeof(int) * 4) == cudaSuccess &&
              cudaMalloc(&g->d_n, sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&g->ticket, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&g->scan_sums, sizeof(int64_t) * pmh_scan_sums_size(Q)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pmh_qgraph_destroy(g);
        return pmh_set_error(PMH_ERR_NOMEM, "graph buffer allocation failed");
    }
    cudaMemset(g->d_n, 0, sizeof(int64_t));
    cudaMemset(g->off, 0, sizeof(int64_t) * (Q + 1));
    cudaStream_t cs;
    PMH_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int U = 4;  // points per lane per round of the walk form
    const int64_t launches0 = g_pmh_launches.load();
    int rc = PMH_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = pmh_set_error(PMH_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    if (rc == PMH_OK && cudaMemsetAsync(g->flags, 0, sizeof(int) * 4, cs) != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "capture memset failed");
    if (rc == PMH_OK)
        rc = pmh_launch_prep(ctx->sm_count, g->xy, g->off, Q, g->d_n, max_vertices, g->bbox, g->area2,
                             g->flags, cs);
    if (rc == PMH_OK)
        rc = pmh_launch_slabs_fixed(ctx, g->xy, g->off, Q, g->d_n, g->slab_info, g->slab_sizes,
                                    g->slab_sums, g->slab_ptr, g->cap_ptr, g->slab_cursor, g->slab_edges,
                                    g->cap_edges, cs);
    if (rc == PMH_OK)
        rc = pmh_launch_sign_unified(ctx, U, g->xy, g->off, g->bbox, g->area2, g->slab_info, g->slab_ptr,
                                     g->slab_edges, nullptr, Q, Q, 0, g->d_n, g->flags, &g->P, sidx,
                                     g->ticket, g->hashes, nullptr, cs);
    if (rc == PMH_OK)
        rc = pmh_launch_query(index, g->hashes, Q, g->d_n, g->counts, nullptr, nullptr, 0, g->join_stage,
                              g->cap, g->flags, false, cs);
    if (rc == PMH_OK) rc = pmh_exclusive_scan_i64(ctx, g->counts, g->row_ptr, Q, cs, g->scan_sums);
    if (rc == PMH_OK)
        rc = pmh_launch_query(index, g->hashes, Q, g->d_n, nullptr, g->row_ptr, g->cand, g->cap,
                              g->join_stage, g->cap, g->flags, true, cs);
    if (rc == PMH_OK)
        rc = pmh_launch_agree(ctx, g->hashes, index->hashes, g->row_ptr, g->cand, Q, g->cap, &g->P,
                              g->count16, nullptr, g->flags, cs);
    if (rc == PMH_OK && S == 0)
        rc = pmh_launch_topm(g->row_ptr, g->cand, g->count16, nullptr, Q, m, K, g->top_ids, g->top_n,
                             g->flags, cs);
    if (S > 0) {
        // learned form (A7): the top-S by count rescored by the MLP; the top-m by score go on
        // to refinement
        if (rc == PMH_OK)
            rc = pmh_launch_topm(g->row_ptr, g->cand, g->count16, nullptr, Q, S, K, g->sl_ids, g->sl_n,
                                 g->flags, cs);
        if (rc == PMH_OK)
            rc = pmh_launch_poly_feat(ctx->sm_count, g->area2, g->off, Q, g->d_n, g->qfeat, cs);
        const FeatSrc qf{g->qfeat, g->bbox, g->area2}, pf{db->feat, db->bbox, db->area2};
        if (g->fused_select) {
            // features, scores and the top-m by score in one launch
            if (rc == PMH_OK)
                rc = pmh_launch_rerank_select(g->rerank, g->hashes, index->hashes, g->sl_ids, g->sl_n, Q,
                                              g->d_n, S, m, &g->P, qf, pf, g->top_ids, g->top_n, g->flags, cs);
        } else {
            // other shortlist lengths: compact lists, feature rows, forward pass, top-m
            if (rc == PMH_OK)
                rc = pmh_launch_lists_to_csr(ctx, g->sl_ids, g->sl_n, Q, S, g->d_n, g->sl_counts, g->sl_sums,
                                             g->sl_row_ptr, g->sl_cand, cs);
            if (rc == PMH_OK)
                rc = pmh_launch_agree_features(ctx, g->hashes, index->hashes, g->sl_row_ptr, g->sl_cand, Q,
                                               Q * S, &g->P, nullptr, nullptr, g->feat, qf, pf, g->flags, cs);
            if (rc == PMH_OK)
                rc = pmh_launch_rerank_forward(g->rerank, g->feat, Q * S, g->score, g->flags, cs);
            if (rc == PMH_OK)
                rc = pmh_launch_topm(g->sl_row_ptr, g->sl_cand, nullptr, g->score, Q, m, 0, g->top_ids,
                                     g->top_n, g->flags, cs);
        }
    }
    if (rc == PMH_OK && k > 0)
        rc = pmh_launch_refine_topk(ctx, g->xy, g->off, g->area2, g->bbox, db, g->top_ids, g->top_n, Q, g->d_n, m,
                                    k, g->jv, g->ticket + 1, g->ref_ids, g->ref_j, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (rc == PMH_OK && e != cudaSuccess)
        rc = pmh_set_error(PMH_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    g->graph = graph;
    g->kernels = g_pmh_launches.load() - launches0;
    g_pmh_launches.fetch_sub(g->kernels);  // captured, not launched: counted per replay
    if (rc == PMH_OK) {
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) rc = pmh_set_error(PMH_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    cudaStreamDestroy(cs);
    if (rc != PMH_OK) {
        cudaGetLastError();
        pmh_qgraph_destroy(g);
        return rc;
    }
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    *out = g;
    return PMH_OK;
}

extern "C" int pmh_qgraph_run(pmh_qgraph g, const int32_t* xy, const int64_t* offsets,
                              int64_t n_queries, int64_t n_vertices, int host_memory, void* stream)
{
    if (!g) return pmh_set_error(PMH_ERR_ARG, "null graph");
    PMH_TRY(pmh_check_device(g->ctx));
    if (g->sidx_cell && g->ctx->sindex.cell[0] != g->sidx_cell)
        return pmh_set_error(PMH_ERR_STATE, "the context's stream index was rebuilt for other "
                                            "parameters since the graph was captured: recreate the graph");
    if (n_queries < 0 || n_queries > g->maxQ || n_vertices < 0 || n_vertices > g->maxV ||
        (n_queries > 0 && (!xy || !offsets)))
        return pmh_set_error(PMH_ERR_RANGE, "batch of %lld queries / %lld vertices exceeds the "
                             "graph's %lld / %lld", (long long)n_queries, (long long)n_vertices,
                             (long long)g->maxQ, (long long)g->maxV);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyKind kind = host_memory ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (n_vertices > 0) PMH_CUDA_TRY(cudaMemcpyAsync(g->xy, xy, sizeof(int2) * n_vertices, kind, s));
    if (n_queries > 0)
        PMH_CUDA_TRY(cudaMemcpyAsync(g->off, offsets, sizeof(int64_t) * (n_queries + 1), kind, s));
    set_batch_kernel<<<1, 1, 0, s>>>(g->d_n, n_queries);
    PMH_LAUNCHED("set_batch_kernel");
    PMH_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    g_pmh_launches.fetch_add(g->kernels);  // the kernels the graph holds
    return PMH_OK;
}

extern "C" int pmh_qgraph_outputs(pmh_qgraph g, uint32_t** d_hashes, int64_t** d_row_ptr,
                                  int32_t** d_cand, uint16_t** d_count, int32_t** d_top_ids,
                                  int32_t** d_top_n)
{
    if (!g) return pmh_set_error(PMH_ERR_ARG, "null graph");
    if (d_hashes) *d_hashes = g->hashes;
    if (d_row_ptr) *d_row_ptr = g->row_ptr;
    if (d_cand) *d_cand = g->cand;
    if (d_count) *d_count = g->count16;
    if (d_top_ids) *d_top_ids = g->top_ids;
    if (d_top_n) *d_top_n = g->top_n;
    return PMH_OK;
}

extern "C" int pmh_qgraph_refined(pmh_qgraph g, int32_t** d_top_ids, double** d_top_j)
{
    if (!g) return pmh_set_error(PMH_ERR_ARG, "null graph");
    if (g->k == 0) return pmh_set_error(PMH_ERR_STATE, "the graph was captured without refinement");
    if (d_top_ids) *d_top_ids = g->ref_ids;
    if (d_top_j) *d_top_j = g->ref_j;
    return PMH_OK;
}

extern "C" int pmh_qgraph_status(pmh_qgraph g, int* h_flags, int64_t* h_total, void* stream)
{
    if (!g) return pmh_set_error(PMH_ERR_ARG, "null graph");
    PMH_TRY(pmh_check_device(g->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    int flags = 0;
    int64_t total = 0;
    PMH_CUDA_TRY(cudaMemcpyAsync(&flags, g->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaMemcpyAsync(&total, g->row_ptr + g->maxQ, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_flags) *h_flags = flags;
    if (h_total) *h_total = total;
    return PMH_OK;
}

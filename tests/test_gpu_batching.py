"""GPU parity of the batching pieces (A9): signing-kernel variants and their autotuner,
and the CUDA-graph query pipeline, against the plain calls and the CPU oracle."""
import numpy as np
import pytest
import torch

from paper_2511_16576_gb300 import synth
from test_gpu_parity import DEV, from_polys, u32, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2511_16576_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def test_every_sign_variant_is_bit_exact(B, ctx, orc):
    db = synth.star_polygons(400, 21, (3, 600), "loguniform", (1e-3, 3e-2))
    P = B.make_params(96, 12, 1 << 24)
    ref = orc.sign(db.xy, db.offsets, P.seed, 96, P.T, nthreads=8)
    polys = upload(B, ctx, db)
    for v in range(B.SIGN_VARIANTS):
        B.sign_set_variant(ctx, v)
        assert np.array_equal(u32(B.minhash_sign(ctx, polys, P)), ref), B.sign_variant_info(v)
    B.sign_set_variant(ctx, -1)


def test_autotune_picks_a_variant(B, ctx, tmp_path, monkeypatch):
    monkeypatch.setattr(B, "_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    w = synth.WORKLOADS["scale"]
    db = synth.make_database(w, 4000)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed)
    polys = upload(B, ctx, db)
    best, ms = B.sign_autotune(ctx, polys, P, cache_key="test")
    assert 0 <= best < B.SIGN_VARIANTS and len(ms) == B.SIGN_VARIANTS
    assert ms[best] == min(ms) and all(t > 0 for t in ms)
    # a cached choice is applied without timing
    best2, ms2 = B.sign_autotune(ctx, polys, P, cache_key="test")
    assert best2 == best and ms2 == ms
    B.sign_set_variant(ctx, -1)


@pytest.fixture(scope="module")
def small_index(B, ctx):
    w = synth.WORKLOADS["small"]
    db = synth.make_database(w)
    qs = synth.make_queries(w, db, 300)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    index = B.lsh_build(ctx, h, P)
    return w, db, qs, P, h, index


@pytest.fixture(scope="module")
def small_index_k128(B, ctx):
    """The small workload signed with K = 128 in 16 bands of 8 (the feature rows' fast
    group bits: one lane's four hashes per group; the block join)."""
    w = synth.WORKLOADS["small"]
    db = synth.make_database(w)
    qs = synth.make_queries(w, db, 300)
    P = B.make_params(128, 16, w.T, w.seed, w.lsh_seed)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    index = B.lsh_build(ctx, h, P)
    return w, db, qs, P, h, index


def plain_outputs(B, ctx, qs, P, h, index, m):
    qh = B.minhash_sign(ctx, upload(B, ctx, qs), P)
    row_ptr, cand = B.lsh_query(ctx, index, qh)
    count, _ = B.jaccard_estimate(ctx, qh, h, row_ptr, cand, P, bandmask=False)
    ids, nn = B.topm(ctx, row_ptr, cand, count, m)
    return qh, row_ptr, cand, count, ids, nn


def test_query_graph_matches_plain_calls(B, ctx, orc, small_index):
    w, db, qs, P, h, index = small_index
    m = 8
    g = B.QueryGraph(ctx, index, max_queries=128, max_vertices=20000, cand_capacity=200000, m=m)
    try:
        for lo, n, host in ((0, 1, False), (1, 7, False), (8, 100, True), (108, 128, False),
                            (0, 0, False)):
            batch = qs.subset(np.arange(lo, lo + n))
            if host:
                g.run(batch.xy, batch.offsets)
            else:
                g.run(torch.from_numpy(batch.xy).to(DEV), torch.from_numpy(batch.offsets).to(DEV))
            flags, total = g.status()
            assert flags == 0
            if n == 0:
                assert total == 0
                continue
            qh, row_ptr, cand, count, ids, nn = plain_outputs(B, ctx, batch, P, h, index, m)
            assert torch.equal(g.hashes[:n], qh)
            assert torch.equal(g.row_ptr[:n + 1], row_ptr) and total == cand.numel()
            assert (g.row_ptr[n:] == total).all()
            assert torch.equal(g.cand[:total], cand)
            assert torch.equal(g.count[:total], count)
            assert torch.equal(g.top_ids[:n], ids) and torch.equal(g.top_n[:n], nn)
            # and against the oracle on this batch
            qh_ref = orc.sign(batch.xy, batch.offsets, w.seed, w.K, w.T)
            assert np.array_equal(u32(g.hashes[:n]), qh_ref)
    finally:
        g.close()


def test_query_graph_overflow_invalid_and_recovery(B, ctx, small_index):
    w, db, qs, P, h, index = small_index
    g = B.QueryGraph(ctx, index, max_queries=64, max_vertices=10000, cand_capacity=3, m=4)
    try:
        batch = qs.subset(np.arange(0, 64))
        g.run(torch.from_numpy(batch.xy).to(DEV), torch.from_numpy(batch.offsets).to(DEV))
        flags, total = g.status()
        assert flags == 8 and total > 3
        assert (g.top_n[:64] == 0).all() and (g.top_ids[:64] == -1).all()
        bad = from_polys([[[0, 0], [5, 0], [0, 5]], [[1, 1], [2, 2]]])
        g.run(bad.xy, bad.offsets)
        flags, total = g.status()
        assert flags == 2 and total == 0   # fewer than 3 vertices
        one = qs.subset([0])
        g.run(one.xy, one.offsets)
        flags, total = g.status()
        assert flags in (0, 8)
        if flags == 0:
            qh, row_ptr, cand, count, ids, nn = plain_outputs(B, ctx, one, P, h, index, 4)
            assert torch.equal(g.top_ids[:1], ids)
        with pytest.raises(B.PmhError):
            big = qs.subset(np.arange(0, 65))
            g.run(big.xy, big.offsets)
    finally:
        g.close()


def test_query_graph_indexed_large_polygons_refined(B, ctx, orc):
    """The graph with the stream index, query polygons of every size class (staged ones,
    fractal polygons of up to 3,000 vertices with slab lists, a comb whose slab lists do not
    fit the graph's fixed buffers, two 5,000-6,000-vertex polygons signed without a
    coverage mask) and exact refinement to the top-10: hashes equal the oracle's, the join,
    counts and top-m equal the plain calls, and the refined top-10 equals pmh_refine_topk
    on the same lists."""
    from test_gpu_parity import comb
    db = synth.star_polygons(3000, 41, (8, 3000), "loguniform", (1e-4, 2e-2), fractal=True,
                             comonotone=True)
    K, bands, m, k = 64, 16, 16, 10
    P = B.make_params(K, bands, 1 << 24, flags=B.FLAG_STREAM_INDEX)
    dbp = upload(B, ctx, db)
    h = B.minhash_sign(ctx, dbp, P)
    index = B.lsh_build(ctx, h, P)
    qs = synth.perturbed_queries(db, 150, 77)
    big = synth.star_polygons(2, 43, (5000, 6000), "uniform", (1e-2, 2e-2), fractal=True)
    polys = [qs.poly(i) for i in range(qs.n)]
    polys[5] = comb(5000, 5000, 500, 10, 10, 5000, 100)
    polys[40], polys[41] = big.poly(0), big.poly(1)
    allq = from_polys(polys)
    g = B.QueryGraph(ctx, index, max_queries=160, max_vertices=allq.n_vertices,
                     cand_capacity=2_000_000, m=m, db=dbp, k=k)
    try:
        for lo, n, host in ((0, 1, False), (0, 33, True), (33, 117, False), (0, 150, False),
                            (3, 0, False)):
            batch = allq.subset(np.arange(lo, lo + n))
            if host:
                g.run(batch.xy, batch.offsets)
            else:
                g.run(torch.from_numpy(batch.xy).to(DEV), torch.from_numpy(batch.offsets).to(DEV))
            flags, total = g.status()
            assert flags == 0
            if n == 0:
                assert total == 0
                continue
            qp = upload(B, ctx, batch)
            qh, row_ptr, cand, count, ids, nn = plain_outputs(B, ctx, batch, P, h, index, m)
            assert torch.equal(g.hashes[:n], qh)
            assert np.array_equal(u32(qh), orc.sign(batch.xy, batch.offsets, P.seed, K, P.T,
                                                   nthreads=16))
            assert torch.equal(g.row_ptr[:n + 1], row_ptr) and total == cand.numel()
            assert torch.equal(g.cand[:total], cand) and torch.equal(g.count[:total], count)
            assert torch.equal(g.top_ids[:n], ids) and torch.equal(g.top_n[:n], nn)
            ti, tj = B.refine_topk(ctx, qp, dbp, ids, nn, k)
            assert torch.equal(g.ref_ids[:n], ti) and torch.equal(g.ref_j[:n], tj)
            assert (ti[:, 0] >= 0).sum() > n // 2   # most queries find their source
            qp.close()
    finally:
        g.close()
        index.close()
        dbp.close()


@pytest.mark.parametrize("which,m,S,fused", [("small_index", 6, 16, True), ("small_index", 6, 24, False),
                                             ("small_index", 10, 32, True), ("small_index", 10, 32, False),
                                             ("small_index", 32, 32, True), ("small_index", 4, 4, True),
                                             ("small_index_k128", 10, 32, True), ("small_index_k128", 10, 32, False),
                                             ("small_index_k128", 4, 4, True), ("small_index_k128", 17, 64, True)])
def test_query_graph_learned_form_matches_plain_calls(B, ctx, request, which, m, S, fused):
    """With a reranker the graph's top-m are the m best by predicted Jaccard among the
    shortlist by agreement count: equal to the same chain of plain calls (shortlist top-S,
    compact lists, features, forward, top-m by score, refinement): the graph's separate
    launches, and its fused selection launch (features, tcgen05 scores and ranking in one
    kernel; shortlists dividing 128); K = 32 and K = 128 (its fast group bits)."""
    w, db, qs, P, h, index = request.getfixturevalue(which)
    dbp = upload(B, ctx, db)
    r = B.Reranker(ctx, seed=5)
    k = 4
    g = B.QueryGraph(ctx, index, max_queries=128, max_vertices=20000, cand_capacity=200000, m=m,
                     db=dbp, k=k, rerank=r, shortlist=S, fused_select=fused)
    try:
        for lo, n in ((0, 1), (1, 90), (0, 128)):
            batch = qs.subset(np.arange(lo, lo + n))
            g.run(torch.from_numpy(batch.xy).to(DEV), torch.from_numpy(batch.offsets).to(DEV))
            assert g.status()[0] == 0
            qp = upload(B, ctx, batch)
            qh, row_ptr, cand, count, _, _ = plain_outputs(B, ctx, batch, P, h, index, m)
            ids1, nn1 = B.topm(ctx, row_ptr, cand, count, S)
            rp2, c2 = B.lists_to_csr(ctx, ids1, nn1)
            feat = B.rerank_features(ctx, qp, dbp, qh, h, rp2, c2, P)
            score = r.forward(feat)
            ids, nn = B.topm(ctx, rp2, c2, None, m, score=score)
            assert torch.equal(g.top_ids[:n], ids) and torch.equal(g.top_n[:n], nn)
            ti, tj = B.refine_topk(ctx, qp, dbp, ids, nn, k)
            assert torch.equal(g.ref_ids[:n], ti) and torch.equal(g.ref_j[:n], tj)
            qp.close()
    finally:
        g.close()
        r.close()
        dbp.close()


def test_query_graph_fused_select_needs_a_dividing_shortlist(B, ctx, small_index):
    """The fused selection takes 128 / S whole queries per tile: other shortlists are
    refused before anything is allocated."""
    w, db, qs, P, h, index = small_index
    dbp = upload(B, ctx, db)
    r = B.Reranker(ctx, seed=5)
    try:
        with pytest.raises(B.PmhError):
            B.QueryGraph(ctx, index, max_queries=16, max_vertices=5000, cand_capacity=10000, m=6, db=dbp, k=4,
                         rerank=r, shortlist=24, fused_select=True)
    finally:
        r.close()
        dbp.close()


def test_reload_and_rebuild_in_place_keep_a_graph_valid(B, ctx, orc):
    """pmh_poly_reload and pmh_lsh_rebuild keep their buffers: a graph captured on the set
    and its index answers for the new data exactly like a fresh upload and build."""
    w = synth.WORKLOADS["small"]
    a = synth.make_database(w)
    # new data with a's vertex counts (a translated copy), so that it fits a's buffers
    shift = np.array([137, -211])
    b = synth.PolySet(a.xy + shift.astype(np.int32), a.offsets.copy(), a.centre + shift, a.rbar)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, B.FLAG_STREAM_INDEX)
    qs = synth.make_queries(w, b, 60)
    dbp = upload(B, ctx, a)
    h = B.minhash_sign(ctx, dbp, P)
    index = B.lsh_build(ctx, h, P)
    g = B.QueryGraph(ctx, index, max_queries=64, max_vertices=10000, cand_capacity=100000, m=8,
                     db=dbp, k=5)
    try:
        B.poly_reload(dbp, torch.from_numpy(b.xy).to(DEV), torch.from_numpy(b.offsets).to(DEV))
        B.minhash_sign(ctx, dbp, P, out=h)
        B.lsh_rebuild(ctx, index, h)
        assert np.array_equal(u32(h), orc.sign(b.xy, b.offsets, w.seed, w.K, w.T, nthreads=8))
        g.run(torch.from_numpy(qs.xy).to(DEV), torch.from_numpy(qs.offsets).to(DEV))
        assert g.status()[0] == 0
        fresh = upload(B, ctx, b)
        h2 = B.minhash_sign(ctx, fresh, P)
        index2 = B.lsh_build(ctx, h2, P)
        qh, row_ptr, cand, count, ids, nn = plain_outputs(B, ctx, qs, P, h2, index2, 8)
        assert torch.equal(g.top_ids[:qs.n], ids) and torch.equal(g.top_n[:qs.n], nn)
        qp = upload(B, ctx, qs)
        ti, tj = B.refine_topk(ctx, qp, fresh, ids, nn, 5)
        assert torch.equal(g.ref_ids[:qs.n], ti) and torch.equal(g.ref_j[:qs.n], tj)
        # the sizes must match the set's
        with pytest.raises(B.PmhError):
            B.poly_reload(dbp, torch.from_numpy(b.xy[:-1]).to(DEV),
                          torch.from_numpy(b.offsets).to(DEV))
        index2.close()
        fresh.close()
        qp.close()
    finally:
        g.close()
        index.close()
        dbp.close()

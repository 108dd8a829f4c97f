"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

Hashes, band keys, candidate sets, agreement counts, band bits and top-m lists must be
bit-identical; exact Jaccard (fp64, different algorithms on the two sides) agrees to a
relative 1e-9.
"""
import numpy as np
import pytest
import torch

from paper_2511_16576_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
SEED = 0x5EED
T24 = 1 << 24


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


def upload(B, ctx, ps):
    return B.poly_upload(ctx, torch.from_numpy(ps.xy).to(DEV), torch.from_numpy(ps.offsets).to(DEV))


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def from_polys(polys):
    xy = np.concatenate([np.asarray(p, np.int32).reshape(-1, 2) for p in polys])
    off = np.zeros(len(polys) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    return synth.PolySet(xy, off, np.zeros((len(polys), 2), np.int64), np.ones(len(polys)))


@pytest.fixture(scope="module")
def small():
    w = synth.WORKLOADS["small"]
    db = synth.make_database(w)
    qs = synth.make_queries(w, db)
    return w, db, qs


def test_prep_bbox_and_area(B, ctx, orc, small):
    _, db, _ = small
    P = upload(B, ctx, db)
    bbox, area2 = P.prep()
    bbox, area2 = bbox.cpu().numpy(), area2.cpu().numpy()
    for i in range(db.n):
        ref = orc.bbox(db.poly(i))
        assert list(bbox[i]) == [max(ref[0], 0), max(ref[1], 0), min(ref[2], 65536), min(ref[3], 65536)]
        assert area2[i] == orc.area2(db.poly(i))


def test_upload_rejects_bad_input(B, ctx):
    ps = from_polys([[[0, 0], [5, 0], [0, 5]], [[1, 1], [2, 2]]])   # second has 2 vertices
    with pytest.raises(B.PmhError):
        upload(B, ctx, ps)
    ps = from_polys([[[0, 0], [5, 0], [0, 1 << 22]]])
    with pytest.raises(B.PmhError):
        upload(B, ctx, ps)


FLAGS = [0, 1, 3]   # 1 = signing through the stream index, 2 = through coverage masks


@pytest.mark.parametrize("flags", FLAGS)
def test_sign_small_bit_exact(B, ctx, orc, small, flags):
    w, db, qs = small
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, flags)
    h = u32(B.minhash_sign(ctx, upload(B, ctx, db), P))
    ref = orc.sign(db.xy, db.offsets, w.seed, w.K, w.T, nthreads=8)
    assert np.array_equal(h, ref)


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("K,T", [(40, 1 << 24), (32, 100), (7, 3000), (64, 1), (32, 70000)])
def test_sign_ragged_K_and_cap(B, ctx, orc, K, T, flags):
    db = synth.star_polygons(300, 11, (3, 40), "loguniform", (2e-6, 2e-2))
    P = B.make_params(K, 1, T, flags=flags)
    h = u32(B.minhash_sign(ctx, upload(B, ctx, db), P))
    ref = orc.sign(db.xy, db.offsets, SEED, K, T, nthreads=8)
    assert np.array_equal(h, ref)


@pytest.mark.parametrize("flags", FLAGS)
def test_sign_edge_cases(B, ctx, orc, flags):
    polys = [
        [[0, 0], [65536, 0], [65536, 65536], [0, 65536]],          # covers the domain: all 0
        [[-100, -100], [70000, -50], [70000, 70000], [-90, 70000]],  # beyond the domain
        [[5, 5], [9, 5], [7, 5]],                                   # zero area: all T
        [[60000, 60000], [70000, 60000], [70000, 70000]],            # partly outside
        [[1000, 1000], [1010, 1000], [1010, 1010], [1000, 1010]][::-1],  # clockwise square
        [[200, 200], [300, 200], [300, 250], [250, 250], [250, 300], [200, 300]],  # L shape
    ]
    # a 2000-vertex star exercises the global-memory edge path (> 256 vertices)
    big = synth.star_polygons(1, 5, (2000, 2000), "uniform", (2e-3, 2e-3))
    polys.append(big.poly(0))
    ps = from_polys(polys)
    # tiny polygons (indexed form, including walks resumed past the index) and a thin sliver
    polys.append([[30000, 30000], [30040, 30000], [30040, 30030], [30000, 30030]])
    polys.append([[100, 100], [160, 103], [120, 150]])
    polys.append([[5000, 5000], [9000, 5001], [9000, 5003], [5000, 5002]])
    ps = from_polys(polys)
    K, T = 64, 200000
    P = B.make_params(K, 1, T, flags=flags)
    h = u32(B.minhash_sign(ctx, upload(B, ctx, ps), P))
    ref = orc.sign(ps.xy, ps.offsets, SEED, K, T)
    assert np.array_equal(h, ref)
    assert (h[0] == 0).all() and (h[2] == T).all()


def comb(x0, y0, teeth, tw, gap, height, base):
    """A comb: a bar of the given base height with `teeth` upward teeth (4 * teeth vertices)."""
    xe = x0 + teeth * (tw + gap) - gap
    pts = [[x0, y0], [xe, y0]]
    for t in reversed(range(teeth)):
        xl = x0 + t * (tw + gap)
        pts += [[xl + tw, y0 + base + height], [xl, y0 + base + height]]
        if t > 0:
            pts += [[xl, y0 + base], [xl - gap, y0 + base]]
    return pts


@pytest.mark.parametrize("flags", FLAGS)
def test_sign_indexed_form_paths(B, ctx, orc, flags):
    """Polygons signed through the stream index: a comb whose 240 vertices need more
    slab references than a warp stages (one slab of every edge instead), more hashes
    than one pass holds (K = 300), tiny boxes whose walks resume past the index, boxes
    on the coarser grid levels, and caps below and above the index limits."""
    polys = [comb(20000, 20000, 60, 10, 10, 1000, 50), comb(40000, 7000, 30, 12, 8, 400, 5)]
    tiny = synth.star_polygons(40, 29, (3, 256), "loguniform", (1e-6, 3e-4))
    polys += [tiny.poly(i) for i in range(tiny.n)]
    # boxes that span many fine cells take the coarser grid levels
    mid = synth.star_polygons(30, 37, (16, 256), "loguniform", (2e-3, 8e-3))
    polys += [mid.poly(i) for i in range(mid.n)]
    ps = from_polys(polys)
    for K, T in [(300, 1 << 24), (33, 5000), (64, 70000)]:
        P = B.make_params(K, 1, T, flags=flags)
        h = u32(B.minhash_sign(ctx, upload(B, ctx, ps), P))
        ref = orc.sign(ps.xy, ps.offsets, SEED, K, T, nthreads=16)
        assert np.array_equal(h, ref), (K, T)


def test_sign_kernel_report(B, ctx):
    """Per-kernel events and work counts: with the stream index one launch (the unified
    kernel) signs every polygon and its counts are pmh_sign_work's; without it the walk
    kernel does; events cover exactly the calls made with timing on."""
    db = synth.star_polygons(3000, 31, (16, 400), "loguniform", (1e-4, 1e-2))
    dbp = upload(B, ctx, db)
    for flags, ran, idle in ((B.FLAG_STREAM_INDEX, "unified", "walk"), (0, "walk", "unified")):
        P = B.make_params(64, 8, T24, flags=flags)
        B.sign_report(ctx)
        B.sign_timing(ctx, True)
        h1 = B.minhash_sign(ctx, dbp, P)
        h2 = B.minhash_sign(ctx, dbp, P)
        B.sign_timing(ctx, False)
        B.minhash_sign(ctx, dbp, P)
        rep = B.sign_report(ctx)
        assert rep["calls"] == 2 and torch.equal(h1, h2)
        assert rep[ran]["ms"] > 0 and rep[idle]["ms"] < rep[ran]["ms"] * 0.05
        total = B.sign_work(ctx)
        for k, v in total.items():
            assert v == rep[ran]["work"][k] and rep[idle]["work"][k] == 0, k
        assert rep[ran]["work"]["walk_points"] > 0 and rep[ran]["work"]["edge_tests"] > 0
        if flags:
            assert rep[ran]["work"]["cells"] > 0 and rep[ran]["work"]["mask_decisions"] > 0
        assert B.sign_report(ctx)["calls"] == 0


@pytest.fixture(scope="module")
def scale_db():
    return synth.make_database(synth.WORKLOADS["scale"])


@pytest.mark.parametrize("flags", FLAGS)
def test_sign_scale_workload_sampled(B, ctx, orc, scale_db, flags):
    """The 1,000,000-polygon, K = 128 workload in the benchmark's launch, sampled rows."""
    w = synth.WORKLOADS["scale"]
    db = scale_db
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, flags)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(db.n, 96, replace=False))
    rows = np.concatenate([rows, [0, db.n - 1]])
    sub = db.subset(rows)
    ref = orc.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=16)
    assert np.array_equal(u32(h[torch.from_numpy(rows).to(DEV)]), ref)
    # property at every size: all hashes below the cap (every polygon is large enough)
    assert int(torch.max(h.view(torch.int32))) < w.T


def test_sign_combined_workload_sampled(B, ctx, orc):
    """The 10,000,000-polygon, K = 128 workload (8-1,024 vertices, area fractions down to
    1e-5, whose walks run past the shallow index levels into the deep one) in the
    benchmark's launch: sampled rows of every size class bit-exact, and every hash below
    the cap."""
    w = synth.WORKLOADS["combined"]
    db = synth.make_database(w)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, B.FLAG_STREAM_INDEX)
    dbp = upload(B, ctx, db)
    h = B.minhash_sign(ctx, dbp, P)
    n = np.diff(db.offsets)
    rng = np.random.default_rng(3)
    # rows of each class: the smallest polygons (deep index level), staged ones, large ones
    order = np.argsort(n, kind="stable")
    rows = np.concatenate([order[:16], rng.choice(db.n, 32, replace=False), order[-16:],
                           [0, db.n - 1]])
    rows = np.unique(rows)
    sub = db.subset(rows)
    ref = orc.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=16)
    assert np.array_equal(u32(h[torch.from_numpy(rows).to(DEV)]), ref)
    assert int(torch.max(h.view(torch.int32))) < w.T
    dbp.close()
    del h


def test_band_keys_bit_exact(B, ctx, orc):
    rng = np.random.default_rng(3)
    for K, b in ((32, 8), (128, 16), (256, 32), (128, 128)):
        h = rng.integers(0, 5000, size=(500, K)).astype(np.uint32)
        h[rng.random(h.shape) < 0.02] = T24
        P = B.make_params(K, b)
        keys = B.band_keys(ctx, torch.from_numpy(h.view(np.int32)).to(DEV), P)
        ref = orc.band_keys(h, b, K // b, T24, 0x15A)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref)


def run_pipeline(B, ctx, w, db, qs, K, b, T):
    P = B.make_params(K, b, T, w.seed, w.lsh_seed)
    dbp, qp = upload(B, ctx, db), upload(B, ctx, qs)
    h = B.minhash_sign(ctx, dbp, P)
    qh = B.minhash_sign(ctx, qp, P)
    index = B.lsh_build(ctx, h, P)
    row_ptr, cand = B.lsh_query(ctx, index, qh)
    return P, dbp, qp, h, qh, index, row_ptr, cand


@pytest.mark.parametrize("K,b,T", [(32, 8, T24), (32, 16, T24), (32, 32, 60), (128, 128, T24)])
def test_candidates_bit_exact(B, ctx, orc, small, K, b, T):
    w, db, qs = small
    P, dbp, qp, h, qh, index, row_ptr, cand = run_pipeline(B, ctx, w, db, qs, K, b, T)
    h_ref = orc.sign(db.xy, db.offsets, w.seed, K, T, nthreads=8)
    qh_ref = orc.sign(qs.xy, qs.offsets, w.seed, K, T, nthreads=8)
    assert np.array_equal(u32(h), h_ref) and np.array_equal(u32(qh), qh_ref)
    rp_ref, cand_ref = orc.candidates(qh_ref, h_ref, b, K // b, T)
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
    assert np.array_equal(cand.cpu().numpy(), cand_ref)
    # agreement counts and band bits
    count, mask = B.jaccard_estimate(ctx, qh, h, row_ptr, cand, P)
    c_ref, m_ref = orc.agree(qh_ref, h_ref, b, K // b, T, rp_ref, cand_ref)
    assert np.array_equal(count.cpu().numpy().view(np.uint16), c_ref)
    assert np.array_equal(mask.cpu().numpy().view(np.uint32), m_ref)
    # top-m by (count desc, id asc)
    for m in (1, 5, 64):
        ids, nn = B.topm(ctx, row_ptr, cand, count, m)
        ids_ref, nn_ref = orc.topm_by_count(rp_ref, cand_ref, c_ref, m)
        assert np.array_equal(ids.cpu().numpy(), ids_ref)
        assert np.array_equal(nn.cpu().numpy(), nn_ref)


def test_query_capacity_and_empty(B, ctx, small):
    w, db, qs = small
    P, dbp, qp, h, qh, index, row_ptr, cand = run_pipeline(B, ctx, w, db, qs, 32, 8, T24)
    total = cand.numel()
    assert total > 0
    with pytest.raises(B.PmhError) as ei:
        B.lsh_query(ctx, index, qh, capacity=total - 1)
    assert ei.value.code == B.PMH_ERR_CAPACITY
    rp0, c0 = B.lsh_query(ctx, index, qh[:0])
    assert rp0.cpu().tolist() == [0] and c0.numel() == 0


def disjoint_triple(ps):
    """Three polygons with pairwise disjoint bounding boxes: no stream point lies in two of
    them, so no hash (and no band) of one equals the other's."""
    box = np.array([[p[:, 0].min(), p[:, 1].min(), p[:, 0].max(), p[:, 1].max()]
                    for p in (ps.poly(i) for i in range(ps.n))])

    def apart(i, j):
        a, b = box[i], box[j]
        return a[2] < b[0] or b[2] < a[0] or a[3] < b[1] or b[3] < a[1]
    for i in range(ps.n):
        for j in range(i + 1, ps.n):
            if not apart(i, j):
                continue
            for k in range(j + 1, ps.n):
                if apart(i, k) and apart(j, k):
                    return i, j, k
    raise AssertionError("no three disjoint polygons")


@pytest.mark.parametrize("bands", [8, 16, 32])
def test_candidates_of_long_rows_bit_exact(B, ctx, orc, bands):
    """Candidate rows of every length the join meets: queries with 3,000, 6,000 and
    20,000 exact duplicates in a database of 29,997 polygons -- rows of at most 3,997
    (the small shared-memory set of 4,096 distinct candidates), of 6,000 to 6,997 (the
    large set of 16,384) and above 20,000 (two id-range passes of the large set) --
    among ordinary rows; bit-exact against the oracle's bucket definition.  Three
    fills: a second call that counts again and joins every row (no capacity given),
    the staged rows copied into place (capacity given), and a lone 6,000-row query
    whose row does not fit the staging pool (4,096 ids per query) and is joined again."""
    w = synth.WORKLOADS["small"]
    base = synth.make_database(w)
    a, b, c = disjoint_triple(base)
    rest = np.setdiff1d(np.arange(base.n), [a, b, c])
    ids = np.concatenate([np.full(3000, a), np.full(6000, b), np.full(20000, c), rest])
    db, qs = base.subset(ids), base.subset(np.concatenate([[a, b, c], rest[:21]]))
    K = 32
    P = B.make_params(K, bands, w.T, w.seed, w.lsh_seed)
    h_ref = orc.sign(db.xy, db.offsets, w.seed, K, w.T, nthreads=8)
    qh_ref = orc.sign(qs.xy, qs.offsets, w.seed, K, w.T, nthreads=8)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    qh = B.minhash_sign(ctx, upload(B, ctx, qs), P)
    assert np.array_equal(u32(h), h_ref) and np.array_equal(u32(qh), qh_ref)
    index = B.lsh_build(ctx, h, P)
    row_ptr, cand = B.lsh_query(ctx, index, qh)
    rp_ref, cand_ref = orc.candidates(qh_ref, h_ref, bands, K // bands, w.T)
    lens = np.diff(rp_ref)
    assert 3000 <= lens[0] <= 3997 and 6000 <= lens[1] <= 6997 and lens[2] >= 20000
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
    assert np.array_equal(cand.cpu().numpy(), cand_ref)
    row_ptr, cand = B.lsh_query(ctx, index, qh, capacity=int(rp_ref[-1]))
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
    assert np.array_equal(cand.cpu().numpy(), cand_ref)
    if bands >= 16:
        row_ptr, cand = B.lsh_query(ctx, index, qh[1:2].contiguous(), capacity=int(lens[1]))
        assert np.array_equal(cand.cpu().numpy(), cand_ref[rp_ref[1]:rp_ref[2]])
        # the query graph: its staging pool holds the candidate capacity
        g = B.QueryGraph(ctx, index, qs.n, qs.xy.shape[0], int(rp_ref[-1]) + 1024, 8)
        try:
            g.run(torch.from_numpy(qs.xy).to(DEV), torch.from_numpy(qs.offsets).to(DEV))
            assert g.status()[0] == 0
            assert np.array_equal(g.row_ptr[:qs.n + 1].cpu().numpy(), rp_ref)
            assert np.array_equal(g.cand[:int(rp_ref[-1])].cpu().numpy(), cand_ref)
        finally:
            g.close()
    index.close()


def test_agreement_on_dense_pairs_with_sentinels(B, ctx, orc):
    rng = np.random.default_rng(9)
    for K, b in ((128, 16), (256, 32), (36, 4), (30, 5)):
        ph = rng.integers(0, 3, size=(40, K)).astype(np.uint32)
        ph[rng.random(ph.shape) < 0.1] = T24
        qh = ph[:7].copy()
        qh[:, ::3] = rng.integers(0, 3, size=qh[:, ::3].shape)
        row_ptr = np.arange(8, dtype=np.int64) * 40
        cand = np.tile(np.arange(40, dtype=np.int32), 7)
        P = B.make_params(K, b)
        count, mask = B.jaccard_estimate(ctx, torch.from_numpy(qh.view(np.int32)).to(DEV),
                                         torch.from_numpy(ph.view(np.int32)).to(DEV),
                                         torch.from_numpy(row_ptr).to(DEV),
                                         torch.from_numpy(cand).to(DEV), P)
        c_ref, m_ref = orc.agree(qh, ph, b, K // b, T24, row_ptr, cand)
        assert np.array_equal(count.cpu().numpy().view(np.uint16), c_ref)
        assert np.array_equal(mask.cpu().numpy().view(np.uint32), m_ref)


def test_topm_large_rows_and_scores(B, ctx):
    rng = np.random.default_rng(4)
    # rows 5..8 for the count form's threshold selection: one long tie (every count
    # equal: the gathered set passes 2,048 and the row takes the merge form), mostly
    # zero counts (the threshold is 0 for large m), counts up to 4,096, and a tie at
    # the threshold that still fits the gathered set
    lens = [0, 1, 7, 3000, 5000, 6000, 4000, 2500, 2300]
    row_ptr = np.zeros(len(lens) + 1, np.int64)
    row_ptr[1:] = np.cumsum(lens)
    E = int(row_ptr[-1])
    cand = rng.integers(0, 1 << 30, E).astype(np.int32)
    count = rng.integers(0, 40, E).astype(np.uint16)
    r = lambda q: slice(row_ptr[q], row_ptr[q + 1])
    count[r(5)] = 7
    count[r(6)] = 0
    count[r(6)][rng.choice(4000, 30, replace=False)] = rng.integers(1, 128, 30).astype(np.uint16)
    count[r(7)] = rng.integers(0, 4097, 2500).astype(np.uint16)
    count[r(8)] = np.where(rng.random(2300) < 0.5, 3, rng.integers(0, 3, 2300)).astype(np.uint16)
    count[r(8)][:5] = 9
    score = rng.random(E).astype(np.float32)
    score[::5] = score[1::5][: len(score[::5])] if E > 5 else score[::5]
    t = lambda a: torch.from_numpy(a).to(DEV)
    for m in (1, 10, 1024):
        ids, nn = B.topm(ctx, t(row_ptr), t(cand), t(count.view(np.int16)), m)
        ids_s, nn_s = B.topm(ctx, t(row_ptr), t(cand), t(count.view(np.int16)), m, score=t(score))
        for q in range(len(lens)):
            seg = slice(row_ptr[q], row_ptr[q + 1])
            exp = [c for _, c in sorted(zip(-count[seg].astype(int), cand[seg]))][:m]
            exp_s = [c for _, c in sorted(zip(-score[seg].astype(np.float64), cand[seg]))][:m]
            got = ids.cpu().numpy()[q]
            got_s = ids_s.cpu().numpy()[q]
            assert list(got[:len(exp)]) == exp and (got[len(exp):] == -1).all()
            assert list(got_s[:len(exp_s)]) == exp_s
            assert nn.cpu().numpy()[q] == len(exp)


def test_pair_jaccard_matches_oracle(B, ctx, orc, small):
    w, db, qs = small
    dbp, qp = upload(B, ctx, db), upload(B, ctx, qs)
    rng = np.random.default_rng(2)
    qid = np.repeat(np.arange(qs.n, dtype=np.int32), 6)
    pid = np.empty_like(qid)
    for q in range(qs.n):
        pid[q * 6] = qs.source[q]
        pid[q * 6 + 1:q * 6 + 6] = rng.integers(0, db.n, 5)
    j = B.pair_jaccard(ctx, qp, dbp, torch.from_numpy(qid).to(DEV), torch.from_numpy(pid).to(DEV))
    j = j.cpu().numpy()
    for e in range(len(qid)):
        ref = orc.jaccard(qs.poly(int(qid[e])), db.poly(int(pid[e])))
        assert abs(j[e] - ref) <= 1e-9 * max(ref, 1e-300) + 1e-12, (e, j[e], ref)


def test_pair_jaccard_degenerate_contacts(B, ctx, orc):
    """Identical polygons, shared edges, vertex-on-edge, nested, golden closed forms."""
    import os
    from test_oracle_area import load_golden
    pairs = [(a, b) for _, a, b, _, _ in load_golden()]
    sq = [[0, 0], [10, 0], [10, 10], [0, 10]]
    pairs += [
        (sq, sq),
        (sq, [[10, 0], [20, 0], [20, 10], [10, 10]]),            # shared edge, disjoint
        (sq, [[5, 0], [15, 0], [15, 10], [5, 10]]),              # overlapping collinear edges
        (sq, [[5, 5], [10, 0], [10, 10]]),                       # vertex on edge, inside
        (sq, [[0, 0], [10, 10], [0, 10]]),                       # diagonal half
        (sq[::-1], [[2, 2], [8, 2], [8, 8], [2, 8]]),            # orientation mix, nested
        ([[0, 0], [4, 0], [4, 2], [2, 2], [2, 4], [0, 4]], [[2, 2], [6, 2], [6, 6], [2, 6]]),
    ]
    ps_a = from_polys([a for a, _ in pairs])
    ps_b = from_polys([b for _, b in pairs])
    pa, pb = upload(B, ctx, ps_a), upload(B, ctx, ps_b)
    idx = torch.arange(len(pairs), dtype=torch.int32, device=DEV)
    j = B.pair_jaccard(ctx, pa, pb, idx, idx).cpu().numpy()
    for e, (a, b) in enumerate(pairs):
        ref = orc.jaccard(np.asarray(a, np.int32), np.asarray(b, np.int32))
        assert abs(j[e] - ref) <= 1e-12 + 1e-9 * ref, (e, j[e], ref)


@pytest.mark.parametrize("m,k", [(32, 10), (7, 3), (1, 1)])
def test_refine_topk_matches_oracle(B, ctx, orc, small, m, k):
    """Refined top-k of top-m lists (work items of a few list slots of one query: m = 7
    leaves a short last item; lists shorter than m leave empty slots)."""
    w, db, qs = small
    P, dbp, qp, h, qh, index, row_ptr, cand = run_pipeline(B, ctx, w, db, qs, 32, 32, T24)
    count, _ = B.jaccard_estimate(ctx, qh, h, row_ptr, cand, P)
    ids, nn = B.topm(ctx, row_ptr, cand, count, m)
    top_ids, top_j = B.refine_topk(ctx, qp, dbp, ids, nn, k)
    ids, nn = ids.cpu().numpy(), nn.cpu().numpy()
    top_ids, top_j = top_ids.cpu().numpy(), top_j.cpu().numpy()
    for q in range(qs.n):
        js = [(orc.jaccard(qs.poly(q), db.poly(int(p))), int(p)) for p in ids[q, :nn[q]]]
        js.sort(key=lambda t: (-t[0], t[1]))
        exp = js[:k]
        for s, (jr, pr) in enumerate(exp):
            assert abs(top_j[q, s] - jr) <= 1e-9 * max(jr, 1e-300) + 1e-12
            # ids equal unless the Jaccard values tie within rounding
            if top_ids[q, s] != pr:
                assert abs(orc.jaccard(qs.poly(q), db.poly(int(top_ids[q, s]))) - jr) < 1e-9
        assert (top_ids[q, len(exp):] == -1).all()


@pytest.mark.parametrize("flags", FLAGS)
def test_sign_batching_workload_sampled(B, ctx, orc, flags):
    """Fractal coastline-like polygons with 4..65,536 vertices (slab-index edge path), K = 256."""
    w = synth.WORKLOADS["batching"]
    db = synth.make_database(w, 600)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, flags)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    n = np.diff(db.offsets)
    order = np.argsort(n)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([order[-10:], order[:4], rng.choice(db.n, 10, replace=False)]))
    sub = db.subset(rows)
    ref = orc.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=16)
    assert n[rows].max() > 30000
    assert np.array_equal(u32(h[torch.from_numpy(rows).to(DEV)]), ref)


def test_sign_slab_index_degenerate(B, ctx, orc):
    """Large polygons whose slab lists hold horizontal edges, vertical runs and spikes."""
    polys = []
    # comb: 300 teeth, horizontal edges on every tooth, vertices on slab boundaries
    pts = [[1000, 1000]]
    for i in range(300):
        x = 1000 + 20 * i
        pts += [[x, 3000], [x + 10, 3000], [x + 10, 1200], [x + 20, 1200]]
    pts += [[1000 + 20 * 300, 1000]]
    polys.append(pts)
    # a 65,536-vertex fractal star
    big = synth.star_polygons(1, 17, (65536, 65536), "uniform", (5e-2, 5e-2), fractal=True)
    polys.append(big.poly(0))
    # a 1,000-vertex regular polygon (many slabs, short edges)
    ang = np.arange(1000) * 2 * np.pi / 1000
    polys.append(np.stack([np.rint(30000 + 9000 * np.cos(ang)),
                           np.rint(30000 + 9000 * np.sin(ang))], 1).astype(np.int32))
    ps = from_polys(polys)
    K, T = 64, 1 << 24
    P = B.make_params(K, 1, T)
    h = u32(B.minhash_sign(ctx, upload(B, ctx, ps), P))
    ref = orc.sign(ps.xy, ps.offsets, SEED, K, T, nthreads=4)
    assert np.array_equal(h, ref)


def test_bbox_join_and_brute_force_truth(B, ctx, orc, small):
    """Brute-force candidates = bbox overlaps (oracle MBRs); exact top-10 = oracle Jaccard."""
    from paper_2511_16576_gb300 import evaluate as ev
    w, db, qs = small
    dbp, qp = upload(B, ctx, db), upload(B, ctx, qs)
    row_ptr, cand = B.bbox_join(ctx, qp, dbp)
    rp, cd = row_ptr.cpu().numpy(), cand.cpu().numpy()
    qb = np.array([orc.bbox(qs.poly(i)) for i in range(qs.n)])
    pb = np.array([orc.bbox(db.poly(i)) for i in range(db.n)])
    for q in range(qs.n):
        a = qb[q]
        exp = np.nonzero((a[0] < pb[:, 2]) & (pb[:, 0] < a[2]) & (a[1] < pb[:, 3]) & (pb[:, 1] < a[3]))[0]
        assert list(cd[rp[q]:rp[q + 1]]) == list(exp)
    truth = ev.brute_force_topk(ctx, qp, dbp, 10)
    for q in range(0, qs.n, 7):
        js = [(orc.jaccard(qs.poly(q), db.poly(int(p))), int(p)) for p in cd[rp[q]:rp[q + 1]]]
        js = sorted([t for t in js if t[0] > 0], key=lambda t: (-t[0], t[1]))[:10]
        assert truth.n_pos[q] == len(js)
        for s, (jr, pr) in enumerate(js):
            assert abs(truth.j[q, s] - jr) <= 1e-9 * jr + 1e-12
    # the exact search finds itself: recall of the truth against itself is 1
    assert ev.recall_at_k(truth.ids, truth.j, truth, 10) == 1.0


def test_pair_jaccard_large_polygons(B, ctx, orc):
    """Pairs too large for the warp's shared slice (global-memory path of the refinement)."""
    big = synth.star_polygons(3, 23, (300, 1500), "uniform", (2e-3, 4e-3), fractal=True)
    qs = synth.perturbed_queries(big, 3, 24)
    dbp, qp = upload(B, ctx, big), upload(B, ctx, qs)
    qid = np.array([0, 1, 2, 0], np.int32)
    pid = np.array([int(qs.source[0]), int(qs.source[1]), int(qs.source[2]), 1], np.int32)
    j = B.pair_jaccard(ctx, qp, dbp, torch.from_numpy(qid).to(DEV), torch.from_numpy(pid).to(DEV))
    j = j.cpu().numpy()
    for e in range(len(qid)):
        ref = orc.jaccard(qs.poly(int(qid[e])), big.poly(int(pid[e])))
        assert abs(j[e] - ref) <= 1e-9 * max(ref, 1e-300) + 1e-12, (e, j[e], ref)
    assert j[0] > 0.5

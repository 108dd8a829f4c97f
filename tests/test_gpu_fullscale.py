"""GPU parity at the full size of the 1,000,000-polygon workload, in the benchmark's
launch configuration, and of the paper's single-hashmap candidate sets.

* every one of the 1.28e8 hashes of the 1,000,000-polygon, K = 128 database equals the
  oracle's (the oracle signs the whole database on the host cores);
* the bucket index of those signatures at 16 bands x 8 rows and at 32 x 4 (16M and 32M
  entries through the multi-block radix sort and scan): for sampled queries, the
  candidate CSR, agreement counts, band bits and top-32 lists equal the oracle's O(Q N b)
  definitions over the whole database;
* the paper's configuration (Sec. 3.2 after Theorem 1, Sec. 5.2): one hashmap keyed on
  the m-hash code (b = 1, r = m, m = 1..5) on a paper-shaped centred set, candidate sets
  equal the oracle's.
"""
import os

import numpy as np
import pytest
import torch

from paper_2511_16576_gb300 import synth
from test_gpu_parity import DEV, u32, upload

pytestmark = pytest.mark.gpu
THREADS = max(1, os.cpu_count() or 1)


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


@pytest.fixture(scope="module")
def scale(B, ctx, orc):
    w = synth.WORKLOADS["scale"]
    db = synth.make_database(w)
    qs = synth.make_queries(w, db)
    h_ref = orc.sign(db.xy, db.offsets, w.seed, w.K, w.T, nthreads=THREADS)
    P = B.make_params(w.K, w.bands, w.T, w.seed, w.lsh_seed, B.FLAG_STREAM_INDEX)
    dbp = upload(B, ctx, db)
    h = B.minhash_sign(ctx, dbp, P)
    yield w, db, qs, h_ref, h
    dbp.close()


def test_sign_every_hash_of_the_full_database(scale):
    w, db, qs, h_ref, h = scale
    got = u32(h)
    assert got.shape == h_ref.shape == (1_000_000, 128)
    bad = np.nonzero((got != h_ref).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first {bad[:5]}"


@pytest.mark.parametrize("bands", [16, 32])
def test_index_at_full_size_matches_oracle(B, ctx, orc, scale, bands):
    w, db, qs, h_ref, h = scale
    P = B.make_params(w.K, bands, w.T, w.seed, w.lsh_seed, B.FLAG_STREAM_INDEX)
    index = B.lsh_build(ctx, h, P)
    rng = np.random.default_rng(bands)
    rows = np.sort(rng.choice(qs.n, 48, replace=False))
    sub = qs.subset(rows)
    qh_ref = orc.sign(sub.xy, sub.offsets, w.seed, w.K, w.T, nthreads=THREADS)
    qh = B.minhash_sign(ctx, upload(B, ctx, sub), P)
    assert np.array_equal(u32(qh), qh_ref)
    row_ptr, cand = B.lsh_query(ctx, index, qh)
    rp_ref, cand_ref = orc.candidates(qh_ref, h_ref, bands, w.K // bands, w.T)
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
    assert np.array_equal(cand.cpu().numpy(), cand_ref)
    assert len(cand_ref) > 48   # the sample has candidates
    count, mask = B.jaccard_estimate(ctx, qh, h, row_ptr, cand, P)
    cnt_ref, mask_ref = orc.agree(qh_ref, h_ref, bands, w.K // bands, w.T, rp_ref, cand_ref)
    assert np.array_equal(count.cpu().numpy().view(np.uint16), cnt_ref)
    assert np.array_equal(mask.cpu().numpy().view(np.uint32), mask_ref)
    ids, nn = B.topm(ctx, row_ptr, cand, count, 32)
    ids_ref, nn_ref = orc.topm_by_count(rp_ref, cand_ref, cnt_ref, 32)
    assert np.array_equal(ids.cpu().numpy(), ids_ref) and np.array_equal(nn.cpu().numpy(), nn_ref)
    index.close()


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_paper_single_hashmap_candidates(B, ctx, orc, m):
    """b = 1 band of r = m rows on centred paper-shaped polygons (Sec. 3.1 preparation):
    the bucket of the whole m-hash code, exactly as the oracle's definition."""
    db = synth.paper_shaped(20_000, 12.0, seed=7)
    qs = synth.paper_queries(db, 40, seed=107)
    P = B.make_params(m, 1, 1 << 24, flags=B.FLAG_STREAM_INDEX)
    h_ref = orc.sign(db.xy, db.offsets, P.seed, m, P.T, nthreads=THREADS)
    qh_ref = orc.sign(qs.xy, qs.offsets, P.seed, m, P.T, nthreads=THREADS)
    h = B.minhash_sign(ctx, upload(B, ctx, db), P)
    qh = B.minhash_sign(ctx, upload(B, ctx, qs), P)
    assert np.array_equal(u32(h), h_ref) and np.array_equal(u32(qh), qh_ref)
    index = B.lsh_build(ctx, h, P)
    row_ptr, cand = B.lsh_query(ctx, index, qh)
    rp_ref, cand_ref = orc.candidates(qh_ref, h_ref, 1, m, P.T)
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref)
    assert np.array_equal(cand.cpu().numpy(), cand_ref)
    # a longer code prunes at least as much: the candidate count falls with m
    assert len(cand_ref) < 40 * db.n
    index.close()

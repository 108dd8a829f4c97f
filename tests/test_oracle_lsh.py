"""Pins of the oracle's band keys, candidate sets, agreement counts and top-m (CPU only).

The paper buckets polygons in a hashmap keyed on their MinHash code (Sec. 3.2 after
Theorem 1; Sec. 5.2, "2 hashmaps" in Sec. 5.3).  With b bands of r rows a polygon is a
candidate of a query iff some band's r-tuple is equal in both and holds no sentinel.
Pins: the band key depends on exactly its own band's rows and on their order; the
sentinel rule; the candidate sets equal those of an independent hashmap construction
(Python dicts keyed on tuples, as the paper describes); agreement counts against
Theorem 1's law.
"""
import math

import numpy as np

from paper_2511_16576_gb300 import synth

T = 1 << 24
LSH_SEED = 0x15A


def test_band_key_depends_on_its_rows_only(orc):
    rng = np.random.default_rng(0)
    K, b, r = 32, 8, 4
    h = rng.integers(0, 5000, size=(64, K)).astype(np.uint32)
    keys = orc.band_keys(h, b, r, T, LSH_SEED)
    for j in range(b):
        for col in range(K):
            h2 = h.copy()
            h2[:, col] += 1
            k2 = orc.band_keys(h2, b, r, T, LSH_SEED)
            changed = np.any(k2[:, j] != keys[:, j])
            assert changed == (j * r <= col < (j + 1) * r)


def test_band_key_is_order_sensitive_and_band_specific(orc):
    h = np.array([[1, 2, 3, 4, 1, 2, 3, 4]], np.uint32)
    k = orc.band_keys(h, 2, 4, T, LSH_SEED)
    # the same tuple in two different bands gives different keys (band index is mixed in)
    assert k[0, 0] != k[0, 1]
    hp = np.array([[2, 1, 3, 4, 1, 2, 3, 4]], np.uint32)
    assert orc.band_keys(hp, 2, 4, T, LSH_SEED)[0, 0] != k[0, 0]
    # a different seed gives different keys
    assert orc.band_keys(h, 2, 4, T, LSH_SEED + 1)[0, 0] != k[0, 0]


def test_band_key_sentinel_and_range(orc):
    rng = np.random.default_rng(1)
    h = rng.integers(0, 1 << 20, size=(20000, 8)).astype(np.uint32)
    h[::7, 3] = T
    keys = orc.band_keys(h, 2, 4, T, LSH_SEED)
    invalid = np.uint64(0xFFFFFFFFFFFFFFFF)
    assert np.all((keys[:, 0] == invalid) == np.any(h[:, 0:4] == T, axis=1))
    assert np.all(keys[:, 1] != invalid)
    # distinct valid tuples give distinct keys (64-bit fingerprints; collisions ~ 2^-35 here)
    valid = keys[:, 1]
    tuples = {tuple(row) for row in h[:, 4:8]}
    assert len(np.unique(valid)) == len(tuples)


def dict_buckets(qh, ph, b, r, cap):
    """The paper's hashmap construction: one dict per band keyed on the r-tuple."""
    maps = [dict() for _ in range(b)]
    for p, row in enumerate(ph):
        for j in range(b):
            t = tuple(int(v) for v in row[j * r:(j + 1) * r])
            if cap in t:
                continue
            maps[j].setdefault(t, []).append(p)
    out = []
    for row in qh:
        s = set()
        for j in range(b):
            t = tuple(int(v) for v in row[j * r:(j + 1) * r])
            if cap in t:
                continue
            s.update(maps[j].get(t, []))
        out.append(sorted(s))
    return out


def test_candidates_equal_hashmap_buckets(orc):
    w = synth.WORKLOADS["small"]
    db = synth.make_database(w, 300)
    qs = synth.make_queries(w, db, 40)
    K, b, r = 16, 8, 2     # short bands so that buckets are populated
    cap = 60   # a small cap exercises the sentinel
    ph = orc.sign(db.xy, db.offsets, w.seed, K, cap)
    qh = orc.sign(qs.xy, qs.offsets, w.seed, K, cap)
    assert (ph == cap).any() and (ph < cap).any()
    row_ptr, cand = orc.candidates(qh, ph, b, r, cap)
    ref = dict_buckets(qh, ph, b, r, cap)
    assert row_ptr[-1] == sum(len(x) for x in ref)
    for q in range(qs.n):
        assert list(cand[row_ptr[q]:row_ptr[q + 1]]) == ref[q]
    # a query is a candidate of itself
    rp2, c2 = orc.candidates(ph[:20], ph, b, r, cap)
    for q in range(20):
        if np.any(np.all(ph[q].reshape(b, r) != cap, axis=1)):
            assert q in set(c2[rp2[q]:rp2[q + 1]])


def test_agreement_counts_and_band_bits(orc):
    rng = np.random.default_rng(5)
    K, b, r = 32, 8, 4
    ph = rng.integers(0, 4, size=(50, K)).astype(np.uint32)
    ph[rng.random(ph.shape) < 0.1] = T
    qh = ph[:10].copy()
    qh[:, ::3] = rng.integers(0, 4, size=qh[:, ::3].shape)
    Q, N = len(qh), len(ph)
    row_ptr = np.arange(Q + 1, dtype=np.int64) * N
    cand = np.tile(np.arange(N, dtype=np.int32), Q)
    count, mask = orc.agree(qh, ph, b, r, T, row_ptr, cand)
    for q in range(Q):
        for p in range(N):
            e = q * N + p
            eq = (qh[q] == ph[p]) & (qh[q] != T)
            assert count[e] == eq.sum()
            bits = sum(1 << j for j in range(b) if eq[j * r:(j + 1) * r].all())
            assert mask[e] == bits


def test_topm_order(orc):
    rng = np.random.default_rng(6)
    row_ptr = np.array([0, 5, 5, 12], np.int64)
    cand = rng.permutation(100)[:12].astype(np.int32)
    count = rng.integers(0, 4, 12).astype(np.uint16)
    ids, n = orc.topm_by_count(row_ptr, cand, count, 4)
    assert list(n) == [4, 0, 4]
    for q in (0, 2):
        seg = sorted(zip(-count[row_ptr[q]:row_ptr[q + 1]].astype(int),
                         cand[row_ptr[q]:row_ptr[q + 1]]))
        assert list(ids[q]) == [int(c) for _, c in seg[:4]]
    assert list(ids[1]) == [-1] * 4


def test_agreement_estimates_jaccard(orc):
    """c/K -> J (Theorem 1) for star pairs: within 4 sd of the lattice Jaccard."""
    K = 2048
    db = synth.star_polygons(4, 61, (10, 30), "uniform", (5e-3, 1e-2))
    qs = synth.perturbed_queries(db, 4, 62)
    ph = orc.sign(db.xy, db.offsets, 0x5EED, K, T, nthreads=4)
    qh = orc.sign(qs.xy, qs.offsets, 0x5EED, K, T, nthreads=4)
    for q in range(qs.n):
        s = int(qs.source[q])
        ca, cb, cab = orc.lattice_pair(qs.poly(q), db.poly(s))
        J = cab / (ca + cb - cab)
        row_ptr = np.array([0, 1], np.int64)
        count, _ = orc.agree(qh[q:q + 1], ph, 1, 1, T, row_ptr, np.array([s], np.int32))
        assert abs(count[0] / K - J) < 4 * math.sqrt(J * (1 - J) / K) + 1e-9

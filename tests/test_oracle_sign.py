"""Pins of the oracle's MinHash (Definition 2, Algorithm 1, Theorems 1 and 2) on the CPU.

h_k(P) = min{ i : point i of stream k is in P } (the min form used in the proof of
Theorem 1), 0-based, capped at T.  Pins: the covering square gives 0; containment gives
h(A) >= h(B); a disjoint split gives h(A u B) = min(h(A), h(B)); the first hit found by an
independent pixel enumeration; hit rates and the geometric law of Theorem 2.
"""
import math

import numpy as np

from paper_2511_16576_gb300 import synth
from test_oracle_membership import crossing_inside, rect

SEED = 0x5EED
T = 1 << 24


def one(poly):
    poly = np.asarray(poly, np.int32)
    return poly, np.array([0, len(poly)], np.int64)


def test_stream_counter_form_equals_sequential(orc):
    for k in (0, 1, 7, 1000):
        x, y = orc.stream_points(SEED, k, 0, 64)
        for i in (0, 1, 5, 63):
            v = orc.stream_value(SEED, k, i)
            assert x[i] == v & 0xFFFF and y[i] == (v >> 16) & 0xFFFF
        x2, y2 = orc.stream_points(SEED, k, 40, 24)
        assert np.array_equal(x2, x[40:]) and np.array_equal(y2, y[40:])


def test_stream_is_uniform_on_the_lattice(orc):
    n = 4_000_000
    x, y = orc.stream_points(SEED, 3, 0, n)
    for v in (x, y, (x >> 8) * 256 + (y >> 8)):
        counts = np.bincount(v.astype(np.int64), minlength=65536)
        e = n / 65536
        chi2 = ((counts - e) ** 2 / e).sum()
        dof = 65535
        assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)
    # consecutive points and neighbouring streams are uncorrelated
    assert abs(np.corrcoef(x[:-1].astype(float), x[1:].astype(float))[0, 1]) < 5e-3
    x2, _ = orc.stream_points(SEED, 4, 0, n)
    assert abs(np.corrcoef(x.astype(float), x2.astype(float))[0, 1]) < 5e-3


def test_covering_square_hashes_to_zero(orc):
    xy, off = one(rect(0, 0, 65536, 65536))
    h = orc.sign(xy, off, SEED, 64, T)
    assert (h == 0).all()


def test_empty_lattice_polygon_hashes_to_sentinel(orc):
    # zero-height polygon and a sliver with no lattice point: never hit
    for p in ([[5, 5], [9, 5], [7, 5]], [[100, 100], [101, 100], [100, 100]]):
        xy, off = one(p)
        assert (orc.sign(xy, off, SEED, 8, T) == T).all()


def test_first_hit_matches_independent_enumeration(orc):
    """First stream index whose point passes an independent crossing-number test."""
    db = synth.star_polygons(6, 21, (6, 30), "uniform", (2e-4, 1e-3))
    for i in range(db.n):
        p = db.poly(i)
        xy, off = one(p)
        h = orc.sign(xy, off, SEED, 16, T)[0]
        x0, y0 = p.min(0)
        x1, y1 = p.max(0)
        for k in range(16):
            x, y = orc.stream_points(SEED, k, 0, 400_000)
            cand = np.nonzero((x >= x0) & (x <= x1) & (y >= y0) & (y <= y1))[0]
            hit = crossing_inside(p, x[cand], y[cand])
            assert hit.any() and h[k] == cand[np.argmax(hit)]


def test_containment_orders_hashes(orc):
    pairs = synth.random_pairs_of_nested(31, 10)
    for inner, outer in pairs:
        hi = orc.sign(*one(inner), SEED, 48, T)[0]
        ho = orc.sign(*one(outer), SEED, 48, T)[0]
        assert (hi >= ho).all()
        # the hash is a hit of the outer polygon too
        assert ((hi == ho) | (hi > ho)).all()


def test_disjoint_split_takes_the_minimum(orc):
    db = synth.star_polygons(8, 33, (8, 24), "uniform", (1e-3, 5e-3))
    for i in range(db.n):
        p = db.poly(i)
        c = db.centre[i]
        j = len(p) // 2
        a = np.vstack([c[None, :], p[:j + 1]]).astype(np.int32)
        b = np.vstack([c[None, :], p[j:], p[:1]]).astype(np.int32)
        hp = orc.sign(*one(p), SEED, 64, T)[0]
        ha = orc.sign(*one(a), SEED, 64, T)[0]
        hb = orc.sign(*one(b), SEED, 64, T)[0]
        assert np.array_equal(hp, np.minimum(ha, hb))
        assert not np.any((ha == hb) & (ha != T))


def test_cap_T_truncates_consistently(orc):
    db = synth.star_polygons(5, 41, (8, 16), "uniform", (1e-4, 2e-4))
    h_big = orc.sign(db.xy, db.offsets, SEED, 32, T)
    for t_small in (50, 1000):
        h = orc.sign(db.xy, db.offsets, SEED, 32, t_small)
        assert np.array_equal(h, np.where(h_big < t_small, h_big, t_small))


def test_hit_rate_matches_lattice_fraction(orc):
    """Each stream point lands in P with probability S_L = |P|_lattice / 2^32 (Eq. spar)."""
    db = synth.star_polygons(3, 51, (12, 30), "uniform", (5e-3, 1e-2))
    M = 1_000_000
    for i in range(db.n):
        p = db.poly(i)
        S = orc.lattice_count(p) / 2.0 ** 32
        x0, y0 = p.min(0)
        x1, y1 = p.max(0)
        total = 0
        for k in range(4):
            x, y = orc.stream_points(SEED, k, 0, M)
            cand = (x >= x0) & (x <= x1) & (y >= y0) & (y <= y1)
            total += int(crossing_inside(p, x[cand], y[cand]).sum())
        n = 4 * M
        assert abs(total - n * S) < 4 * math.sqrt(n * S * (1 - S))


def test_theorem2_mean_and_variance(orc):
    """E[h + 1] = 1/S and Var[h] = (1 - S)/S^2 (Theorem 2, 1-based attempts)."""
    p = np.array([[1000, 1000], [9000, 1500], [8000, 8000], [2000, 7000]], np.int32)
    S = orc.lattice_count(p) / 2.0 ** 32
    K = 4096
    h = orc.sign(*one(p), SEED, K, T)[0].astype(np.float64)
    assert (h < T).all()
    mean = (h + 1).mean()
    sd_mean = math.sqrt((1 - S) / S ** 2 / K)
    assert abs(mean - 1 / S) < 4 * sd_mean
    var = h.var()
    # a geometric law has excess kurtosis ~6, so the sample variance has relative sd
    # ~ sqrt((6 + 2) / K); allow 4 sd
    assert abs(var / ((1 - S) / S ** 2) - 1) < 4 * math.sqrt(8.0 / K)


def test_theorem1_collision_rate_is_lattice_jaccard(orc):
    """Pr[h(P) = h(Q)] = J(P, Q) (Theorem 1) with the lattice areas of this sampler."""
    K = 4096
    a = np.array([[2000, 2000], [9000, 2500], [8500, 9000], [2500, 8000]], np.int32)
    for shift in ([1500, 700], [3000, 2000], [0, 0], [200, -100]):
        b = a + np.array(shift, np.int32)
        ca, cb, cab = orc.lattice_pair(a, b)
        J = cab / (ca + cb - cab)
        ha = orc.sign(*one(a), SEED, K, T)[0]
        hb = orc.sign(*one(b), SEED, K, T)[0]
        rate = np.mean(ha == hb)
        assert abs(rate - J) <= 4 * math.sqrt(max(J * (1 - J), 1e-12) / K) + 1e-12

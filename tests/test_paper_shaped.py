"""Paper-shaped inputs (Sec. 3.1 preprocessing applied at generation): centring on the
centroid, one global MBR mapped onto the lattice.  Pinned against what the preprocessing
fixes: translation invariance, every centred polygon containing the common centre, and
the oracle's hashes of translated copies being equal."""
import numpy as np

import oracle
from paper_2511_16576_gb300 import synth


def test_centroids_of_known_shapes():
    # unit square and a right triangle, in float coordinates
    xy = np.array([[0, 0], [2, 0], [2, 2], [0, 2], [0, 0], [3, 0], [0, 3]], np.float64)
    off = np.array([0, 4, 7])
    c = synth.centroids(xy, off)
    assert np.allclose(c, [[1.0, 1.0], [1.0, 1.0]])


def test_centring_is_translation_invariant():
    db = synth.paper_shaped(300, 9.26, seed=3)
    # float copies of the lattice polygons, each moved by its own offset
    rng = np.random.default_rng(4)
    pid = np.repeat(np.arange(db.n), np.diff(db.offsets))
    shift = rng.uniform(-1e4, 1e4, (db.n, 2))
    a = db.xy.astype(np.float64)
    b = a + shift[pid]
    xa, ya, mbr, o = synth.center_and_quantize(a, db.offsets)
    xb, yb, _, _ = synth.center_and_quantize(b, db.offsets, mbr=mbr)
    d = np.maximum(np.abs(xa - xb), np.abs(ya - yb))
    assert d.max() <= 1 and (d == 0).mean() > 0.999


def test_every_polygon_contains_the_common_centre():
    db = synth.paper_shaped(2000, 12.0, seed=5)
    cx, cy = db.centre[0]
    assert (db.centre == db.centre[0]).all()
    assert np.diff(db.offsets).min() >= 3
    for i in range(0, db.n, 7):
        assert oracle.inside(db.poly(i), int(cx), int(cy))
    c = synth.centroids(db.xy, db.offsets)
    assert np.abs(c - db.centre).max() <= 1.5
    qs = synth.paper_queries(db, 50, seed=6)
    cq = synth.centroids(qs.xy, qs.offsets)
    assert np.abs(cq - qs.centre).max() <= 1.5
    for i in range(qs.n):
        assert oracle.inside(qs.poly(i), int(cx), int(cy))


def test_translated_copies_hash_alike():
    db = synth.paper_shaped(40, 9.26, seed=8)
    pid = np.repeat(np.arange(db.n), np.diff(db.offsets))
    a = db.xy.astype(np.float64)
    b = a + np.array([12345.25, -777.5])[None, :]
    xa, ya, mbr, _ = synth.center_and_quantize(a, db.offsets)
    xb, yb, _, _ = synth.center_and_quantize(b, db.offsets, mbr=mbr)
    same = np.ones(db.n, bool)
    same[pid[(xa != xb) | (ya != yb)]] = False
    pa = np.stack([xa, ya], 1).astype(np.int32)
    pb = np.stack([xb, yb], 1).astype(np.int32)
    ha = oracle.sign(pa, db.offsets, 0x5EED, 8, 1 << 20)
    hb = oracle.sign(pb, db.offsets, 0x5EED, 8, 1 << 20)
    assert same.mean() > 0.9
    assert np.array_equal(ha[same], hb[same])

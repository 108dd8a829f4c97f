"""Pins of the oracle's lattice membership and areas (CPU only).

The paper asks for a "precise point-in-polygon test" (Sec. 3.2, Algorithm 1) and
area-based Jaccard (Sec. 1).  The oracle's membership is the half-open reading: a
lattice point p is in P iff p + (e1, e2), 0 < e2 << e1, lies inside P.  Pins:
closed forms (rectangles, rectilinear polygons whose lattice count equals their area),
the tiling identity (a fan triangulation's pieces add up exactly), invariances, and a
brute-force crossing-number enumeration written independently of the oracle's scanline
spans.
"""
import numpy as np
import pytest

from paper_2511_16576_gb300 import synth


def crossing_inside(poly: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Vectorised even-odd crossing count for p + (e1, e2): edge a->b counts iff
    (ay > py) != (by > py) and the cross product (b-a) x (p-a) is non-zero with the
    sign of (by - ay)."""
    px = px.astype(np.int64)
    py = py.astype(np.int64)
    inside = np.zeros(px.shape, bool)
    n = len(poly)
    for i in range(n):
        ax, ay = int(poly[i, 0]), int(poly[i, 1])
        bx, by = int(poly[(i + 1) % n, 0]), int(poly[(i + 1) % n, 1])
        straddle = (ay > py) != (by > py)
        cross = (bx - ax) * (py - ay) - (px - ax) * (by - ay)
        dy = by - ay
        inside ^= straddle & (cross != 0) & (np.sign(cross) == np.sign(dy))
    return inside


def rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], np.int32)


def test_rectangles_count_their_area(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        x0, x1 = sorted(rng.integers(0, 65537, 2))
        y0, y1 = sorted(rng.integers(0, 65537, 2))
        assert orc.lattice_count(rect(x0, y0, x1, y1)) == (x1 - x0) * (y1 - y0)
        # clockwise order gives the same set
        assert orc.lattice_count(rect(x0, y0, x1, y1)[::-1].copy()) == (x1 - x0) * (y1 - y0)


def test_domain_square_holds_every_lattice_point(orc):
    assert orc.lattice_count(rect(0, 0, 65536, 65536)) == 1 << 32
    assert orc.inside(rect(0, 0, 65536, 65536), 0, 0)
    assert orc.inside(rect(0, 0, 65536, 65536), 65535, 65535)


def random_rectilinear(rng, cells=12, scale=37):
    """Union of unit cells forming a staircase (x-monotone) region, scaled; its boundary is a
    rectilinear polygon."""
    heights = rng.integers(1, cells, size=cells)
    base = rng.integers(0, 3, size=cells)
    # a histogram with bottoms base[i] and tops base[i] + heights[i]; keep it connected by
    # making consecutive columns overlap
    tops = base + heights
    for i in range(1, cells):
        if base[i] >= tops[i - 1]:
            base[i] = tops[i - 1] - 1
        if tops[i] <= base[i - 1]:
            tops[i] = base[i - 1] + 1
    upper = []
    lower = []
    for i in range(cells):
        upper += [(i, tops[i]), (i + 1, tops[i])]
        lower += [(i, base[i]), (i + 1, base[i])]
    pts = lower + upper[::-1]
    # drop collinear duplicates
    out = []
    for p in pts:
        if out and out[-1] == p:
            continue
        out.append(p)
    if out[0] == out[-1]:
        out.pop()
    poly = np.array(out, np.int64) * scale + np.array([1000, 2000])
    return poly.astype(np.int32)


def test_rectilinear_count_equals_shoelace_area(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        p = random_rectilinear(rng)
        a2 = orc.area2(p)
        assert a2 % 2 == 0
        assert orc.lattice_count(p) == abs(a2) // 2


def test_fan_triangulation_tiles_exactly(orc):
    db = synth.star_polygons(40, 7, (5, 40), "uniform", (1e-4, 1e-3))
    for i in range(db.n):
        p = db.poly(i)
        c = db.centre[i]
        total = 0
        for j in range(len(p)):
            tri = np.array([c, p[j], p[(j + 1) % len(p)]], np.int32)
            total += orc.lattice_count(tri)
        assert total == orc.lattice_count(p)


def test_chord_split_adds_exactly(orc):
    db = synth.star_polygons(30, 8, (8, 30), "uniform", (1e-4, 1e-3))
    for i in range(db.n):
        p = db.poly(i)
        c = db.centre[i]
        j = len(p) // 2
        a = np.vstack([c[None, :], p[:j + 1]]).astype(np.int32)
        b = np.vstack([c[None, :], p[j:], p[:1]]).astype(np.int32)
        ca, cb, cab = orc.lattice_pair(a, b)
        assert cab == 0
        assert ca + cb == orc.lattice_count(p)


def test_brute_force_crossing_number_agrees(orc):
    rng = np.random.default_rng(3)
    db = synth.star_polygons(12, 9, (3, 20), "uniform", (2e-7, 2e-6))
    polys = [db.poly(i) for i in range(db.n)]
    # hand-made degenerate cases: horizontal edges, vertices on grid rows, collinear runs
    polys.append(np.array([[10, 10], [20, 10], [20, 15], [15, 15], [15, 20], [10, 20]], np.int32))
    polys.append(np.array([[10, 10], [30, 10], [20, 20]], np.int32))
    polys.append(np.array([[10, 10], [14, 10], [18, 10], [18, 14], [14, 18], [10, 14]], np.int32))
    polys.append(np.array([[5, 5], [25, 9], [12, 30], [9, 18]], np.int32))
    for p in polys:
        x0, y0 = p.min(0) - 2
        x1, y1 = p.max(0) + 2
        gx, gy = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1))
        expect = crossing_inside(p, gx.ravel(), gy.ravel())
        got = np.array([orc.inside(p, int(a), int(b)) for a, b in zip(gx.ravel(), gy.ravel())])
        assert np.array_equal(expect, got)
        assert int(expect.sum()) == orc.lattice_count(p)
    del rng


def test_invariances(orc):
    db = synth.star_polygons(20, 10, (8, 40), "uniform", (1e-4, 1e-3))
    for i in range(db.n):
        p = db.poly(i)
        c = orc.lattice_count(p)
        assert orc.lattice_count(p[::-1].copy()) == c            # orientation
        assert orc.lattice_count(np.roll(p, 3, axis=0)) == c     # start vertex
        assert orc.lattice_count(p + np.array([17, -29], np.int32)) == c  # translation
        # count close to the area: every lattice point owns its unit cell up-right of it,
        # so the difference is bounded by the number of cells the boundary crosses
        perim = np.abs(np.diff(np.vstack([p, p[:1]]), axis=0)).sum()
        assert abs(c - abs(orc.area2(p)) / 2) <= perim + 4


def test_shoelace_area_closed_forms(orc):
    assert orc.area2(rect(0, 0, 4, 3)) == 24
    assert orc.area2(rect(0, 0, 4, 3)[::-1].copy()) == -24
    assert orc.area2(np.array([[0, 0], [8, 0], [0, 8]])) == 64
    assert list(orc.bbox(np.array([[5, 7], [1, 9], [3, -2]]))) == [1, -2, 5, 9]


@pytest.mark.parametrize("scale", [1, 3])
def test_lattice_pair_matches_brute_force(orc, scale):
    a = np.array([[10, 10], [40, 12], [35, 40], [12, 33]], np.int32) * scale
    b = np.array([[20, 5], [50, 25], [25, 45]], np.int32) * scale
    ca, cb, cab = orc.lattice_pair(a, b)
    gx, gy = np.meshgrid(np.arange(0, 60 * scale), np.arange(0, 60 * scale))
    ia = crossing_inside(a, gx.ravel(), gy.ravel())
    ib = crossing_inside(b, gx.ravel(), gy.ravel())
    assert (ca, cb, cab) == (ia.sum(), ib.sum(), (ia & ib).sum())

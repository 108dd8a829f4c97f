"""Pins of the oracle's exact intersection areas and Jaccard similarity (CPU only).

J(A, B) = area(A n B) / area(A u B) (Sec. 1; Theorem 1's right-hand side).  Pins: hand
closed forms (tests/golden), identity, disjointness, containment, symmetry, rectilinear
pairs whose exact area equals the lattice count of the intersection, and convergence of the
lattice Jaccard of scaled copies to the exact value.
"""
import os

import numpy as np
import pytest

from paper_2511_16576_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "jaccard_closed_forms.txt")


def load_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, a, b, inter, j = [s.strip() for s in line.split("|")]
        pa = np.array([[int(v) for v in p.split(",")] for p in a.split(";")], np.int32)
        pb = np.array([[int(v) for v in p.split(",")] for p in b.split(";")], np.int32)
        cases.append((name, pa, pb, float(inter), float(j)))
    return cases


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c[0])
def test_closed_forms(orc, case):
    _, a, b, inter, j = case
    assert orc.intersection_area(a, b) == pytest.approx(inter, rel=1e-12, abs=1e-12)
    assert orc.jaccard(a, b) == pytest.approx(j, rel=1e-12, abs=1e-12)
    # orientation and symmetry do not matter
    assert orc.jaccard(b, a) == pytest.approx(j, rel=1e-12, abs=1e-12)
    assert orc.jaccard(a[::-1].copy(), b) == pytest.approx(j, rel=1e-12, abs=1e-12)


def test_identity_disjoint_containment(orc):
    db = synth.star_polygons(10, 71, (8, 40), "uniform", (1e-4, 1e-3))
    for i in range(db.n):
        p = db.poly(i)
        assert orc.jaccard(p, p) == pytest.approx(1.0, rel=1e-12)
        far = p + np.array([5000, 0], np.int32) if p[:, 0].max() < 60000 else p - 5000
        assert orc.jaccard(p, far) == 0.0
        c = db.centre[i]
        tri = np.array([c, p[0], p[1]], np.int32)
        a_tri = abs(orc.area2(tri)) / 2
        a_p = abs(orc.area2(p)) / 2
        assert orc.intersection_area(tri, p) == pytest.approx(a_tri, rel=1e-12)
        assert orc.jaccard(tri, p) == pytest.approx(a_tri / a_p, rel=1e-12)


def test_symmetry_and_bounds(orc):
    w = synth.WORKLOADS["small"]
    db = synth.make_database(w, 60)
    qs = synth.make_queries(w, db, 30)
    for q in range(qs.n):
        a = qs.poly(q)
        b = db.poly(int(qs.source[q]))
        j1 = orc.jaccard(a, b)
        j2 = orc.jaccard(b, a)
        assert j1 == pytest.approx(j2, rel=1e-12)
        assert 0.5 < j1 <= 1.0   # perturbed copies overlap their source strongly


def random_rect(rng, lo=0, hi=400):
    x0, x1 = sorted(rng.integers(lo, hi, 2))
    y0, y1 = sorted(rng.integers(lo, hi, 2))
    x1 += 1
    y1 += 1
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], np.int32)


def test_rectilinear_pairs_equal_lattice_counts(orc):
    """For rectilinear polygons (and their intersections) the lattice count is the area."""
    from test_oracle_membership import random_rectilinear
    rng = np.random.default_rng(7)
    for _ in range(40):
        a = random_rectilinear(rng, cells=8, scale=11)
        b = random_rectilinear(rng, cells=8, scale=13) + np.array(rng.integers(-60, 60, 2),
                                                                  np.int32)
        ca, cb, cab = orc.lattice_pair(a, b)
        assert orc.intersection_area(a, b) == pytest.approx(cab, abs=1e-9)
        if ca + cb - cab > 0:
            assert orc.jaccard(a, b) == pytest.approx(cab / (ca + cb - cab), rel=1e-12)
    for _ in range(100):
        a, b = random_rect(rng), random_rect(rng)
        ca, cb, cab = orc.lattice_pair(a, b)
        assert orc.intersection_area(a, b) == pytest.approx(cab, abs=1e-9)


def test_lattice_jaccard_converges_under_scaling(orc):
    a = np.array([[3, 1], [17, 4], [14, 15], [6, 12], [1, 7]], np.int64)
    b = np.array([[8, 0], [20, 9], [10, 18], [5, 10]], np.int64)
    exact = orc.jaccard(a, b)
    errs = []
    for s in (16, 64, 256, 1024):
        ca, cb, cab = orc.lattice_pair(a * s, b * s)
        errs.append(abs(cab / (ca + cb - cab) - exact))
        assert orc.jaccard(a * s, b * s) == pytest.approx(exact, rel=1e-12)
    # O(perimeter / s) convergence: the error shrinks with the scale
    assert errs[-1] < 2e-3 and errs[-1] < errs[0]

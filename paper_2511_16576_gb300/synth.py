"""Seeded synthetic polygon workloads.

This module holds no arithmetic of the hashing method: it only draws polygons
and queries.  Both the CUDA path's tests and the CPU oracle's tests take their
inputs from here, so the two never share anything else.

The paper evaluates on UCR-STAR polygon sets (Cemetery, Sports, Parks, Urban
Areas; Sec. 5.1, Table 1) that are not available here; these generators stand
in for them with the shapes the workloads name:

* star polygons: vertices at sorted uniform angles around a centre c, radius
  R * U[1-j, 1+j] with R = sqrt(f * 2^32 / pi) for an area fraction f of the
  65536 x 65536 lattice domain;
* fractal stars: the radius is a midpoint-displacement profile (coastline-like
  boundaries with up to 65,536 vertices);
* queries: perturbed copies of database polygons (rotation, scale, vertex
  jitter about the source centre);
* paper-shaped sets: the vertex-count means and sizes of the paper's four
  sets, prepared as Sec. 3.1 prepares data before hashing (centroid moved to
  the origin, one global MBR mapped onto the lattice).  That preparation is
  done here, at generation time, so that both sides receive the same lattice
  polygons; the hashing itself (Sec. 3.2 on) is not in this module.

Every polygon is rounded to int32 and then made strictly star-shaped around its
(integer) centre by dropping any vertex v_i with (v_i - c) x (v_{i+1} - c) <= 0,
which guarantees a simple polygon.  Layout: ``xy`` int32 [V, 2] interleaved,
``offsets`` int64 [N + 1].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DOMAIN = 65536


@dataclasses.dataclass
class PolySet:
    xy: np.ndarray        # int32 [V, 2]
    offsets: np.ndarray   # int64 [N + 1]
    centre: np.ndarray    # int64 [N, 2]
    rbar: np.ndarray      # float64 [N] nominal radius
    source: np.ndarray | None = None  # int64 [N] database id a query was copied from

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_vertices(self) -> int:
        return int(self.offsets[-1])

    def poly(self, i: int) -> np.ndarray:
        return self.xy[self.offsets[i]:self.offsets[i + 1]]

    def subset(self, ids) -> "PolySet":
        ids = np.asarray(ids, dtype=np.int64)
        counts = self.offsets[ids + 1] - self.offsets[ids]
        offs = np.zeros(len(ids) + 1, np.int64)
        np.cumsum(counts, out=offs[1:])
        idx = np.concatenate([np.arange(self.offsets[i], self.offsets[i + 1]) for i in ids]) \
            if len(ids) else np.zeros(0, np.int64)
        return PolySet(np.ascontiguousarray(self.xy[idx]), offs, self.centre[ids], self.rbar[ids],
                       None if self.source is None else self.source[ids])


def _group_starts(pid: np.ndarray) -> np.ndarray:
    """For a sorted group-id array, the index of the first element of each element's group."""
    n = len(pid)
    first = np.ones(n, bool)
    first[1:] = pid[1:] != pid[:-1]
    starts = np.nonzero(first)[0]
    return starts[np.cumsum(first) - 1]


def _make_star_shaped(x: np.ndarray, y: np.ndarray, pid: np.ndarray, cx: np.ndarray,
                      cy: np.ndarray, n_polys: int, rbar: np.ndarray):
    """Drop vertices until every edge turns strictly counter-clockwise around c."""
    keep = np.ones(len(x), bool)
    active = np.ones(len(x), bool)   # vertices of polygons that may still change
    while True:
        idx = np.nonzero(keep & active)[0]
        if len(idx) == 0:
            break
        p = pid[idx]
        start = _group_starts(p)
        nxt = np.arange(len(idx)) + 1
        last = np.ones(len(idx), bool)
        last[:-1] = p[1:] != p[:-1]
        nxt[last] = start[last]
        ax = x[idx] - cx[p]
        ay = y[idx] - cy[p]
        bx = x[idx[nxt]] - cx[p]
        by = y[idx[nxt]] - cy[p]
        cross = ax * by - bx * ay
        bad = cross <= 0
        if not bad.any():
            break
        keep[idx[bad]] = False
        changed = np.zeros(n_polys, bool)
        changed[p[bad]] = True
        active = changed[pid]
    # polygons left with fewer than 3 vertices become a triangle around c
    counts = np.bincount(pid[keep], minlength=n_polys)
    small = np.nonzero(counts < 3)[0]
    xs, ys, ps = [x[keep]], [y[keep]], [pid[keep]]
    if len(small):
        keep_small = np.isin(pid, small) & keep
        xs, ys, ps = [x[keep & ~keep_small]], [y[keep & ~keep_small]], [pid[keep & ~keep_small]]
        ang = np.array([0.0, 2 * math.pi / 3, 4 * math.pi / 3])
        for s in small:
            r = max(2.0, rbar[s])
            tx = np.rint(cx[s] + r * np.cos(ang)).astype(np.int64)
            ty = np.rint(cy[s] + r * np.sin(ang)).astype(np.int64)
            xs.append(tx)
            ys.append(ty)
            ps.append(np.full(3, s, np.int64))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    p = np.concatenate(ps)
    order = np.argsort(p, kind="stable")
    x, y, p = x[order], y[order], p[order]
    offs = np.zeros(n_polys + 1, np.int64)
    np.cumsum(np.bincount(p, minlength=n_polys), out=offs[1:])
    xy = np.empty((len(x), 2), np.int32)
    xy[:, 0] = x
    xy[:, 1] = y
    return xy, offs


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _fractal_radius(rng, pid: np.ndarray, pos: np.ndarray, n: np.ndarray, amp0: float = 0.25,
                    decay: float = 0.6) -> np.ndarray:
    """Midpoint-displacement radius profile r(t) on t in [0,1), amplitude x decay per level.

    Level l adds 2^l periodic control offsets; a vertex takes the linear interpolation of
    each level's controls at its angle, so the sum is a periodic fractal profile.  A
    polygon only receives the levels its own vertex count can resolve (2^l <= 2n).
    """
    t = pos / n[pid]
    r = np.ones(len(pid))
    levels = int(math.ceil(math.log2(max(int(n.max()), 2)))) + 1
    amp = amp0
    for lev in range(2, levels + 1):
        m = 1 << lev
        elig = np.nonzero(2 * n >= m)[0]
        if len(elig) == 0:
            break
        row = np.full(len(n), -1, np.int64)
        row[elig] = np.arange(len(elig))
        ctrl = rng.uniform(-amp, amp, size=(len(elig), m))
        sel = row[pid] >= 0
        u = t[sel] * m
        i0 = np.floor(u).astype(np.int64) % m
        w = u - np.floor(u)
        i1 = (i0 + 1) % m
        rr = row[pid[sel]]
        r[sel] += (1 - w) * ctrl[rr, i0] + w * ctrl[rr, i1]
        amp *= decay
        if amp < 1e-4:
            break
    return np.clip(r, 0.3, 1.6)


def star_polygons(n_polys: int, seed: int, n_range=(8, 64), n_dist: str = "uniform",
                  f_range=(1e-2, 5e-2), jitter: float = 0.3, fractal: bool = False,
                  comonotone: bool = False) -> PolySet:
    """Seeded star (or fractal-star) polygons on the 65536^2 lattice domain.

    n_dist is "uniform" (integers n_range[0]..n_range[1]) or "loguniform"; the area fraction
    f is log-uniform on f_range; with ``comonotone`` the sorted n are paired with the sorted f
    (both marginals kept) so that polygons with many vertices are also large.
    """
    rng = np.random.default_rng(seed)
    lo, hi = n_range
    if n_dist == "uniform":
        n = rng.integers(lo, hi + 1, size=n_polys)
    else:
        n = np.floor(_loguniform(rng, lo, hi + 1, n_polys)).astype(np.int64)
        n = np.clip(n, lo, hi)
    f = _loguniform(rng, f_range[0], f_range[1], n_polys)
    if comonotone:
        perm = rng.permutation(n_polys)
        n_sorted = np.sort(n)
        f_sorted = np.sort(f)
        n = np.empty_like(n)
        f = np.empty_like(f)
        n[perm] = n_sorted
        f[perm] = f_sorted
    n = n.astype(np.int64)
    rbar = np.sqrt(f * float(DOMAIN) ** 2 / math.pi)
    margin = np.ceil(1.6 * rbar) + 2
    cx = np.rint(rng.uniform(margin, DOMAIN - margin)).astype(np.int64)
    cy = np.rint(rng.uniform(margin, DOMAIN - margin)).astype(np.int64)
    V = int(n.sum())
    pid = np.repeat(np.arange(n_polys, dtype=np.int64), n)
    offs0 = np.zeros(n_polys + 1, np.int64)
    np.cumsum(n, out=offs0[1:])
    pos = np.arange(V, dtype=np.int64) - offs0[pid]
    if fractal:
        # equally spaced angles with a small jitter; radius from the fractal profile
        ang = (pos + rng.uniform(0.1, 0.9, V)) * (2 * math.pi) / n[pid]
        rad = rbar[pid] * _fractal_radius(rng, pid, pos.astype(np.float64), n.astype(np.float64))
    else:
        ang = rng.uniform(0.0, 2 * math.pi, V)
        # sort angles within each polygon
        order = np.lexsort((ang, pid))
        ang = ang[order]
        # a cyclic angular gap of pi or more would leave the centre outside the polygon;
        # such polygons (rare for n >= 8) take stratified angles instead
        nxt_ang = np.empty_like(ang)
        nxt_ang[:-1] = ang[1:]
        nxt_ang[offs0[1:] - 1] = ang[offs0[:-1]] + 2 * math.pi
        gap = nxt_ang - ang
        wide = np.zeros(n_polys, bool)
        wide[pid[gap > 0.75 * math.pi]] = True
        if wide.any():
            sel = wide[pid]
            ang[sel] = (pos[sel] + rng.uniform(0.0, 1.0, int(sel.sum()))) * (2 * math.pi) / n[pid[sel]]
        rad = rbar[pid] * rng.uniform(1.0 - jitter, 1.0 + jitter, V)
    x = np.rint(cx[pid] + rad * np.cos(ang)).astype(np.int64)
    y = np.rint(cy[pid] + rad * np.sin(ang)).astype(np.int64)
    np.clip(x, 0, DOMAIN, out=x)
    np.clip(y, 0, DOMAIN, out=y)
    xy, offs = _make_star_shaped(x, y, pid, cx, cy, n_polys, rbar)
    centre = np.stack([cx, cy], axis=1)
    return PolySet(xy, offs, centre, rbar)


def perturbed_queries(db: PolySet, n_queries: int, seed: int, max_rot_deg: float = 10.0,
                      scale_range=(0.9, 1.1), jitter_frac: float = 0.01) -> PolySet:
    """Perturbed copies of random database polygons (rotation, scale, vertex jitter)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, db.n, size=n_queries)
    theta = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, n_queries))
    scale = rng.uniform(scale_range[0], scale_range[1], n_queries)
    counts = db.offsets[src + 1] - db.offsets[src]
    V = int(counts.sum())
    pid = np.repeat(np.arange(n_queries, dtype=np.int64), counts)
    offs0 = np.zeros(n_queries + 1, np.int64)
    np.cumsum(counts, out=offs0[1:])
    pos = np.arange(V, dtype=np.int64) - offs0[pid]
    vidx = db.offsets[src][pid] + pos
    cx = db.centre[src, 0].astype(np.int64)
    cy = db.centre[src, 1].astype(np.int64)
    rx = db.xy[vidx, 0].astype(np.float64) - cx[pid]
    ry = db.xy[vidx, 1].astype(np.float64) - cy[pid]
    c, s = np.cos(theta)[pid], np.sin(theta)[pid]
    qx = scale[pid] * (c * rx - s * ry)
    qy = scale[pid] * (s * rx + c * ry)
    jit = jitter_frac * db.rbar[src][pid]
    qx += rng.uniform(-1, 1, V) * jit
    qy += rng.uniform(-1, 1, V) * jit
    x = np.clip(np.rint(cx[pid] + qx).astype(np.int64), 0, DOMAIN)
    y = np.clip(np.rint(cy[pid] + qy).astype(np.int64), 0, DOMAIN)
    xy, offs = _make_star_shaped(x, y, pid, cx, cy, n_queries, db.rbar[src])
    return PolySet(xy, offs, np.stack([cx, cy], axis=1), db.rbar[src].copy(), src.astype(np.int64))


# ----------------------------------------------------------------------------
# Paper-shaped sets (Sec. 3.1 preprocessing applied at generation time).
# ----------------------------------------------------------------------------
# Vertex-count means and sizes of the paper's four evaluation sets (Sec. 5.1, Table 1).
PAPER_SETS = {"n9": (149_000, 9.26), "n12": (1_000_000, 12.0), "n95": (11_800, 95.4),
              "n319": (300_000, 319.0)}


def centroids(xy: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Area centroids [N, 2] (float64) of simple polygons given as float or int rings."""
    x = xy[:, 0].astype(np.float64)
    y = xy[:, 1].astype(np.float64)
    n = np.diff(offsets)
    pid = np.repeat(np.arange(len(n)), n)
    nxt = np.arange(len(x)) + 1
    nxt[offsets[1:] - 1] = offsets[:-1]
    cr = x * y[nxt] - x[nxt] * y
    a6 = 3.0 * np.bincount(pid, weights=cr, minlength=len(n))  # 6 * area
    cx = np.bincount(pid, weights=(x + x[nxt]) * cr, minlength=len(n)) / a6
    cy = np.bincount(pid, weights=(y + y[nxt]) * cr, minlength=len(n)) / a6
    return np.stack([cx, cy], axis=1)


def center_and_quantize(xy: np.ndarray, offsets: np.ndarray, mbr=None):
    """Sec. 3.1 preprocessing: move every polygon's centroid to (0, 0), take the global
    MBR of the moved polygons (or the given one), and map it onto the 2^16 lattice
    domain (x and y scaled separately, so that a uniform point of the lattice is a
    uniform point of the MBR).  Returns (int64 x, int64 y, the MBR, the lattice point
    of (0, 0))."""
    c = centroids(xy, offsets)
    pid = np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))
    px = xy[:, 0].astype(np.float64) - c[pid, 0]
    py = xy[:, 1].astype(np.float64) - c[pid, 1]
    if mbr is None:
        mbr = (px.min(), py.min(), px.max(), py.max())
    x0, y0, x1, y1 = mbr
    sx, sy = DOMAIN / (x1 - x0), DOMAIN / (y1 - y0)
    qx = np.clip(np.rint((px - x0) * sx), 0, DOMAIN).astype(np.int64)
    qy = np.clip(np.rint((py - y0) * sy), 0, DOMAIN).astype(np.int64)
    origin = (int(np.rint(-x0 * sx)), int(np.rint(-y0 * sy)))
    return qx, qy, mbr, origin


def paper_shaped(n_polys: int, mean_vertices: float, seed: int, size_ratio: float = 30.0) -> PolySet:
    """Polygons shaped like a paper evaluation set, centred and quantized onto the lattice.

    Vertex counts are 3 + Poisson(mean - 3); radii log-uniform over a ``size_ratio`` span
    (the largest polygons set the global MBR, the smallest are sparse in it); star
    outlines (sorted uniform angles, radius jitter +-30%) in float coordinates, then
    centred on their centroids and mapped onto the lattice by ``center_and_quantize``.
    Every polygon is made star-shaped around the lattice image of (0, 0), so all of
    them contain it, as centred polygons do."""
    rng = np.random.default_rng(seed)
    n = 3 + rng.poisson(max(mean_vertices - 3.0, 0.0), size=n_polys).astype(np.int64)
    r = np.exp(rng.uniform(0.0, math.log(size_ratio), n_polys))
    V = int(n.sum())
    pid = np.repeat(np.arange(n_polys, dtype=np.int64), n)
    offs = np.zeros(n_polys + 1, np.int64)
    np.cumsum(n, out=offs[1:])
    pos = np.arange(V, dtype=np.int64) - offs[pid]
    ang = (pos + rng.uniform(0.05, 0.95, V)) * (2 * math.pi) / n[pid]   # stratified: star-shaped
    rad = r[pid] * rng.uniform(0.7, 1.3, V)
    fxy = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    qx, qy, mbr, origin = center_and_quantize(fxy, offs)
    ox = np.full(n_polys, origin[0], np.int64)
    oy = np.full(n_polys, origin[1], np.int64)
    rbar = r * DOMAIN / (mbr[2] - mbr[0])
    xy, offs2 = _make_star_shaped(qx, qy, pid, ox, oy, n_polys, rbar)
    return PolySet(xy, offs2, np.stack([ox, oy], axis=1), rbar)


def paper_queries(db: PolySet, n_queries: int, seed: int) -> PolySet:
    """Perturbed copies of paper-shaped polygons, centred again on the common lattice
    point (integer shift of each copy's centroid)."""
    qs = perturbed_queries(db, n_queries, seed)
    c = centroids(qs.xy, qs.offsets)
    shift = np.rint(qs.centre - c).astype(np.int64)
    pid = np.repeat(np.arange(qs.n), np.diff(qs.offsets))
    x = np.clip(qs.xy[:, 0].astype(np.int64) + shift[pid, 0], 0, DOMAIN)
    y = np.clip(qs.xy[:, 1].astype(np.int64) + shift[pid, 1], 0, DOMAIN)
    xy, offs = _make_star_shaped(x, y, pid, qs.centre[:, 0], qs.centre[:, 1], qs.n, qs.rbar)
    return PolySet(xy, offs, qs.centre, qs.rbar, qs.source)


# ----------------------------------------------------------------------------
# Named workloads (sizes of the five evaluation configurations).
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_polys: int
    n_range: tuple
    n_dist: str
    f_range: tuple
    K: int
    bands: int
    rows: int
    n_queries: int
    fractal: bool = False
    comonotone: bool = False
    T: int = 1 << 24
    seed: int = 0x5EED
    lsh_seed: int = 0x15A
    gen_seed: int = 1
    query_seed: int = 101


WORKLOADS = {
    "small": Workload("small", 1000, (8, 64), "uniform", (1e-2, 5e-2), 32, 8, 4, 100,
                      gen_seed=1, query_seed=101),
    "scale": Workload("scale", 1_000_000, (16, 256), "loguniform", (1e-4, 1e-2), 128, 16, 8,
                      10_000, gen_seed=2, query_seed=102),
    "batching": Workload("batching", 100_000, (4, 65536), "loguniform", (1e-5, 1e-1), 256, 32, 8,
                         4096, fractal=True, comonotone=True, gen_seed=3, query_seed=103),
    "combined": Workload("combined", 10_000_000, (8, 1024), "loguniform", (1e-5, 1e-2), 128, 16,
                         8, 100_000, fractal=True, comonotone=True, gen_seed=5, query_seed=105),
}


def make_database(w: Workload, n_polys: int | None = None) -> PolySet:
    return star_polygons(n_polys or w.n_polys, w.gen_seed, w.n_range, w.n_dist, w.f_range,
                         fractal=w.fractal, comonotone=w.comonotone)


def make_queries(w: Workload, db: PolySet, n_queries: int | None = None) -> PolySet:
    return perturbed_queries(db, n_queries or w.n_queries, w.query_seed)


def random_pairs_of_nested(seed: int, n: int = 16):
    """(inner, outer) lattice polygons with inner a subset of outer: fan triangles of stars."""
    db = star_polygons(n, seed, (8, 24), "uniform", (1e-3, 1e-2))
    out = []
    for i in range(db.n):
        p = db.poly(i)
        c = db.centre[i]
        j = i % len(p)
        tri = np.array([c, p[j], p[(j + 1) % len(p)]], np.int32)
        out.append((tri, p))
    return out

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

The per-vertex work (angles, radius profiles, rounding, the star-shape filter) runs
in ``synth_gen.c`` on all host cores, with one PCG32 stream per polygon, so that a
10,000,000-polygon set takes seconds; the per-polygon parameters are drawn here.

Every polygon is rounded to int32 and then made strictly star-shaped around its
(integer) centre by dropping any vertex v_i with (v_i - c) x (v_{i+1} - c) <= 0,
which guarantees a simple polygon.  Layout: ``xy`` int32 [V, 2] interleaved,
``offsets`` int64 [N + 1].
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

DOMAIN = 65536

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "synth_gen.c")
_GEN_LIB = os.path.join(_HERE, "_build", "libsynthgen.so")
_gen_lock = threading.Lock()
_gen = None


def build_generator(force: bool = False) -> str:
    """Compile the per-vertex generator (synth_gen.c, plain gcc) into _build/."""
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or \
            os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _GEN_SRC,
                               "-lpthread", "-lm"])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _lib():
    global _gen
    with _gen_lock:
        if _gen is None:
            lib = ctypes.CDLL(build_generator())
            P, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.sg_star_vertices.argtypes = [i64, P, P, P, P, P, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.c_int, P]
            lib.sg_star_vertices.restype = None
            lib.sg_star_filter.argtypes = [i64, P, P, P, P, P, ctypes.c_int, P]
            lib.sg_star_filter.restype = None
            lib.sg_compact.argtypes = [i64, P, P, P]
            lib.sg_compact.restype = None
            _gen = lib
        return _gen


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


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


def _filter_and_pack(xy: np.ndarray, offs0: np.ndarray, cx: np.ndarray, cy: np.ndarray,
                     rbar: np.ndarray):
    """Star-shape filter of every polygon in place (synth_gen.c), then pack the kept
    vertices: returns (xy [V', 2] int32, offsets [N + 1] int64)."""
    n_polys = len(offs0) - 1
    lib = _lib()
    cx, cy, rbar = _c(cx, np.int64), _c(cy, np.int64), _c(rbar, np.float64)
    kept = np.zeros(n_polys, np.int64)
    lib.sg_star_filter(n_polys, offs0.ctypes.data, xy.ctypes.data, cx.ctypes.data, cy.ctypes.data,
                       rbar.ctypes.data, _threads(), kept.ctypes.data)
    offs = np.zeros(n_polys + 1, np.int64)
    np.cumsum(kept, out=offs[1:])
    lib.sg_compact(n_polys, offs0.ctypes.data, offs.ctypes.data, xy.ctypes.data)
    return xy[:offs[-1]], offs


def _make_star_shaped(x: np.ndarray, y: np.ndarray, pid: np.ndarray, cx: np.ndarray,
                      cy: np.ndarray, n_polys: int, rbar: np.ndarray):
    """Drop vertices until every edge turns strictly counter-clockwise around c.

    x, y: vertex coordinates grouped by polygon (pid sorted); polygons left with fewer
    than 3 vertices become a triangle around c."""
    offs0 = np.zeros(n_polys + 1, np.int64)
    np.cumsum(np.bincount(pid, minlength=n_polys), out=offs0[1:])
    xy = np.empty((len(x), 2), np.int32)
    xy[:, 0] = x
    xy[:, 1] = y
    return _filter_and_pack(xy, offs0, cx, cy, rbar)


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


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
    offs0 = np.zeros(n_polys + 1, np.int64)
    np.cumsum(n, out=offs0[1:])
    # per-vertex work in C, one PCG32 stream per polygon seeded from this generator
    vseed = int(rng.integers(0, 1 << 63))
    xy = np.empty((int(offs0[-1]), 2), np.int32)
    _lib().sg_star_vertices(n_polys, n.ctypes.data, offs0.ctypes.data, cx.ctypes.data,
                            cy.ctypes.data, rbar.ctypes.data, float(jitter), int(fractal), vseed,
                            _threads(), xy.ctypes.data)
    xy, offs = _filter_and_pack(xy, offs0, cx, cy, rbar)
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

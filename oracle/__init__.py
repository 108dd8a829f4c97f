"""CPU oracle for the PolyMinHash signature path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles ``oracle.c`` with gcc into
``oracle/_build/liboracle.so`` and wraps it with ctypes + numpy.  It shares no
code with the CUDA library and never imports it.

Paper: PolyMinHash (arXiv 2511.16576).  Each wrapper names the passage the C
routine follows; the readings of the paper are listed at the top of oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, no arch flags)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(src), os.path.getmtime(hdr)))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src,
                               "-lpthread", "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
        sig = {
            "orc_mix64": (u64, [u64]),
            "orc_stream_seed": (u64, [u64, u64]),
            "orc_stream_value": (u64, [u64, u64, u64]),
            "orc_stream_points": (None, [u64, u64, u64, i64, P, P]),
            "orc_inside": (ctypes.c_int, [P, i64, i64, i64]),
            "orc_lattice_count": (i64, [P, i64]),
            "orc_lattice_pair": (ctypes.c_int, [P, i64, P, i64, P, P, P]),
            "orc_area2": (i64, [P, i64]),
            "orc_bbox": (None, [P, i64, P]),
            "orc_sign": (ctypes.c_int, [P, P, i64, u64, u32, u32, P, ctypes.c_int]),
            "orc_sign_work": (ctypes.c_int, [P, P, i64, u64, u32, u32, P, P, P, P]),
            "orc_band_keys": (None, [P, i64, u32, u32, u32, u32, u64, P]),
            "orc_candidates": (i64, [P, i64, P, i64, u32, u32, u32, u32, P, P, i64]),
            "orc_agree": (None, [P, P, u32, u32, u32, u32, P, P, i64, P, P]),
            "orc_topm_by_count": (ctypes.c_int, [P, P, P, i64, i32, P, P]),
            "orc_intersection_area": (ctypes.c_double, [P, i64, P, i64]),
            "orc_jaccard": (ctypes.c_double, [P, i64, P, i64]),
            "orc_bf16_round": (ctypes.c_double, [ctypes.c_double]),
            "orc_mlp_forward_backward": (None, [P, P, i64, i32, i32] + [P] * 14 + [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _poly(xy) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))


# ---------------------------------------------------------------- streams (R1)
def mix64(z: int) -> int:
    return int(_load().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def stream_seed(seed: int, k: int) -> int:
    return int(_load().orc_stream_seed(seed, k))


def stream_value(seed: int, k: int, i: int) -> int:
    return int(_load().orc_stream_value(seed, k, i))


def stream_points(seed: int, k: int, i0: int, count: int):
    """Points i0..i0+count-1 of stream k (Sec. 3.2 seeded uniform sampling)."""
    x = np.empty(count, np.uint32)
    y = np.empty(count, np.uint32)
    _load().orc_stream_points(seed, k, i0, count, _ptr(x), _ptr(y))
    return x, y


# --------------------------------------------------------- membership (R2)
def inside(poly, px: int, py: int) -> bool:
    p = _poly(poly)
    return bool(_load().orc_inside(_ptr(p), len(p), px, py))


def lattice_count(poly) -> int:
    p = _poly(poly)
    return int(_load().orc_lattice_count(_ptr(p), len(p)))


def lattice_pair(a, b):
    """Lattice counts |A|, |B|, |A n B| on [0,65536)^2 (half-open rule R2)."""
    pa, pb = _poly(a), _poly(b)
    ca, cb, cab = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().orc_lattice_pair(_ptr(pa), len(pa), _ptr(pb), len(pb), ctypes.byref(ca),
                                  ctypes.byref(cb), ctypes.byref(cab))
    assert rc == 0
    return ca.value, cb.value, cab.value


def area2(poly) -> int:
    """Twice the signed shoelace area (exact)."""
    p = _poly(poly)
    return int(_load().orc_area2(_ptr(p), len(p)))


def bbox(poly) -> np.ndarray:
    p = _poly(poly)
    out = np.empty(4, np.int32)
    _load().orc_bbox(_ptr(p), len(p), _ptr(out))
    return out


# ------------------------------------------------------ Def. 2 / Alg. 1
def sign(xy, offsets, seed: int, K: int, T: int, nthreads: int = 1) -> np.ndarray:
    """h_k(P) for every polygon and k < K (Definition 2, Algorithm 1, R1-R3)."""
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    out = np.empty((n, K), np.uint32)
    rc = _load().orc_sign(_ptr(xy), _ptr(offsets), n, seed, K, T, _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle sign failed (polygon with < 3 vertices?)")
    return out


def sign_work(xy, offsets, seed: int, K: int, T: int):
    """sign() plus per-polygon work: points drawn, MBR passes, edge tests."""
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    out = np.empty((n, K), np.uint32)
    pts = np.empty(n, np.int64)
    hits = np.empty(n, np.int64)
    edges = np.empty(n, np.int64)
    rc = _load().orc_sign_work(_ptr(xy), _ptr(offsets), n, seed, K, T, _ptr(out), _ptr(pts),
                               _ptr(hits), _ptr(edges))
    if rc != 0:
        raise ValueError("oracle sign failed")
    return out, pts, hits, edges


# --------------------------------------------------------- bands (R4)
def band_keys(hashes, bands: int, rows: int, T: int, lsh_seed: int) -> np.ndarray:
    h = np.ascontiguousarray(hashes, dtype=np.uint32)
    n, K = h.shape
    out = np.empty((n, bands), np.uint64)
    _load().orc_band_keys(_ptr(h), n, K, bands, rows, T, lsh_seed, _ptr(out))
    return out


def candidates(qh, ph, bands: int, rows: int, T: int):
    """CSR (row_ptr, ids) of the band-bucket candidates of every query."""
    qh = np.ascontiguousarray(qh, dtype=np.uint32)
    ph = np.ascontiguousarray(ph, dtype=np.uint32)
    Q, K = qh.shape
    N = ph.shape[0]
    row_ptr = np.empty(Q + 1, np.int64)
    lib = _load()
    dummy = np.empty(1, np.int32)
    total = lib.orc_candidates(_ptr(qh), Q, _ptr(ph), N, K, bands, rows, T, _ptr(row_ptr),
                               _ptr(dummy), 0)
    cand = np.empty(max(total, 1), np.int32)
    lib.orc_candidates(_ptr(qh), Q, _ptr(ph), N, K, bands, rows, T, _ptr(row_ptr), _ptr(cand),
                       total)
    return row_ptr, cand[:total]


def agree(qh, ph, bands: int, rows: int, T: int, row_ptr, cand):
    """Agreement counts and band-match bits of every candidate pair (Thm. 1)."""
    qh = np.ascontiguousarray(qh, dtype=np.uint32)
    ph = np.ascontiguousarray(ph, dtype=np.uint32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    Q, K = qh.shape
    E = int(row_ptr[-1])
    count = np.empty(max(E, 1), np.uint16)
    mask = np.empty(max(E, 1), np.uint32)
    _load().orc_agree(_ptr(qh), _ptr(ph), K, bands, rows, T, _ptr(row_ptr), _ptr(cand), Q,
                      _ptr(count), _ptr(mask))
    return count[:E], mask[:E]


def topm_by_count(row_ptr, cand, count, m: int):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    count = np.ascontiguousarray(count, dtype=np.uint16)
    Q = len(row_ptr) - 1
    ids = np.empty((Q, m), np.int32)
    nn = np.empty(Q, np.int32)
    if len(cand) == 0:
        cand = np.zeros(1, np.int32)
        count = np.zeros(1, np.uint16)
    rc = _load().orc_topm_by_count(_ptr(row_ptr), _ptr(cand), _ptr(count), Q, m, _ptr(ids),
                                   _ptr(nn))
    assert rc == 0
    return ids, nn


# ------------------------------------------------------ exact Jaccard (Sec. 1)
def intersection_area(a, b) -> float:
    pa, pb = _poly(a), _poly(b)
    return float(_load().orc_intersection_area(_ptr(pa), len(pa), _ptr(pb), len(pb)))


def jaccard(a, b) -> float:
    pa, pb = _poly(a), _poly(b)
    return float(_load().orc_jaccard(_ptr(pa), len(pa), _ptr(pb), len(pb)))


# ------------------------------------------------------ reranker reference
def bf16_round(v: float) -> float:
    return float(_load().orc_bf16_round(v))


def mlp_forward_backward(x, y, w1, b1, w2, b2, w3, b3, grads: bool = True, bf16: bool = True):
    """Forward + backward of the 3-layer reranker MLP (fp64, bf16 operands)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    n, d_in = x.shape
    d_h = int(np.asarray(b1).shape[0])
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (w1, b1, w2, b2, w3, b3)]
    pred = np.empty(n, np.float64)
    loss = np.zeros(1, np.float64)
    g = [np.zeros_like(a) for a in arrs] if grads else None
    null = ctypes.c_void_p(0)
    gp = [_ptr(a) for a in g] if grads else [null] * 6
    _load().orc_mlp_forward_backward(_ptr(x), _ptr(y), n, d_in, d_h, *[_ptr(a) for a in arrs],
                                     _ptr(pred), _ptr(loss), *gp, 1 if bf16 else 0)
    return pred, float(loss[0]), g

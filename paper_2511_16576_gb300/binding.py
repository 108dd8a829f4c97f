"""Thin ctypes binding of libpolyminhash.so (the C ABI in include/polyminhash.h).

Argument marshalling only: every step runs in the library's CUDA kernels.  torch
provides device memory and streams.  uint32 / uint16 arrays are carried in int32 /
int16 tensors (same bits); uint64 keys in int64 tensors.  There is no CPU fallback:
if the library is missing or no sm_103 GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpolyminhash.so")
_lib = None

PMH_OK = 0
PMH_ERR_ARG = -1
PMH_ERR_CAPACITY = -3
INVALID_KEY = 0xFFFFFFFFFFFFFFFF


class PmhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"polyminhash error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("K", ctypes.c_uint32), ("T", ctypes.c_uint32),
                ("bands", ctypes.c_uint32), ("rows", ctypes.c_uint32),
                ("lsh_seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class QGraphConfig(ctypes.Structure):
    _fields_ = [("max_queries", ctypes.c_int64), ("max_vertices", ctypes.c_int64),
                ("cand_capacity", ctypes.c_int64), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
                ("db", ctypes.c_void_p), ("rerank", ctypes.c_void_p), ("shortlist", ctypes.c_int32),
                ("options", ctypes.c_int32)]


QGRAPH_FUSED_SELECT = 1


FLAG_STREAM_INDEX = 1
FLAG_COVERAGE_MASK = 2


def make_params(K: int, bands: int, T: int = 1 << 24, seed: int = 0x5EED,
                lsh_seed: int = 0x15A, flags: int = 0) -> Params:
    return Params(seed, K, T, bands, K // bands, lsh_seed, flags, 0)


# entry points: name -> (restype, argtypes)
_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_SIGS = {
    "pmh_last_error": (ctypes.c_char_p, []),
    "pmh_version": (ctypes.c_int, []),
    "pmh_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int]),
    "pmh_destroy": (ctypes.c_int, [_P]),
    "pmh_poly_upload": (ctypes.c_int, [_P, _P, _P, _i64, _i64, ctypes.POINTER(_P), _P]),
    "pmh_poly_upload_host": (ctypes.c_int, [_P, _P, _P, _i64, _i64, ctypes.POINTER(_P), _P]),
    "pmh_poly_reload": (ctypes.c_int, [_P, _P, _P, _i64, _i64, ctypes.c_int, _P]),
    "pmh_polys_info": (ctypes.c_int, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "pmh_polys_prep": (ctypes.c_int, [_P, _P, _P, _P]),
    "pmh_polys_destroy": (ctypes.c_int, [_P]),
    "pmh_minhash_sign": (ctypes.c_int, [_P, _P, ctypes.POINTER(Params), _P, _P]),
    "pmh_band_keys": (ctypes.c_int, [_P, _P, _i64, ctypes.POINTER(Params), _P, _P]),
    "pmh_stream_index_build": (ctypes.c_int, [_P, ctypes.POINTER(Params), _P]),
    "pmh_sign_work": (ctypes.c_int, [_P, _P]),
    "pmh_sign_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmh_sign_count_work": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmh_sign_report": (ctypes.c_int, [_P, _P, _P]),
    "pmh_lsh_build": (ctypes.c_int, [_P, _P, _i64, ctypes.POINTER(Params), ctypes.POINTER(_P), _P]),
    "pmh_lsh_rebuild": (ctypes.c_int, [_P, _P, _P, _i64, _P]),
    "pmh_index_destroy": (ctypes.c_int, [_P]),
    "pmh_lsh_query": (ctypes.c_int, [_P, _P, _P, _i64, _P, _P, _i64, ctypes.POINTER(_i64), _P]),
    "pmh_lsh_query_fill": (ctypes.c_int, [_P, _P, _P, _i64, _P, _P, _i64, _P]),
    "pmh_jaccard_estimate": (ctypes.c_int, [_P, _P, _P, _P, _P, _i64, ctypes.POINTER(Params), _P,
                                            _P, _P]),
    "pmh_topm": (ctypes.c_int, [_P, _P, _P, _P, _P, _i64, _i32, _P, _P, _P]),
    "pmh_refine_topk": (ctypes.c_int, [_P, _P, _P, _P, _P, _i64, _i32, _i32, _P, _P, _P]),
    "pmh_pair_jaccard": (ctypes.c_int, [_P, _P, _P, _P, _P, _i64, _P, _P]),
    "pmh_probe_int_peak": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "pmh_launch_count": (_i64, []),
    "pmh_minhash_sign_noalloc": (ctypes.c_int, [_P, _P, _i64, _i64, ctypes.POINTER(Params), _P,
                                                _P]),
    "pmh_sign_autotune": (ctypes.c_int, [_P, _P, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int),
                                         _P]),
    "pmh_sign_set_variant": (ctypes.c_int, [_P, ctypes.c_int]),
    "pmh_sign_variant_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]),
    "pmh_qgraph_create": (ctypes.c_int, [_P, _P, ctypes.POINTER(QGraphConfig), ctypes.POINTER(_P)]),
    "pmh_qgraph_refined": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "pmh_qgraph_run": (ctypes.c_int, [_P, _P, _P, _i64, _i64, ctypes.c_int, _P]),
    "pmh_qgraph_outputs": (ctypes.c_int, [_P] + [ctypes.POINTER(_P)] * 6),
    "pmh_qgraph_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64), _P]),
    "pmh_qgraph_destroy": (ctypes.c_int, [_P]),
    "pmh_lists_to_csr": (ctypes.c_int, [_P, _P, _P, _i64, _i32, _P, _P, _P]),
    "pmh_bbox_join": (ctypes.c_int, [_P, _P, _P, _P, _P, _i64, ctypes.POINTER(_i64), _P]),
    "pmh_rerank_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "pmh_rerank_destroy": (ctypes.c_int, [_P]),
    "pmh_rerank_set_weights": (ctypes.c_int, [_P, _P]),
    "pmh_rerank_get_weights": (ctypes.c_int, [_P, _P]),
    "pmh_rerank_features": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _i64, ctypes.POINTER(Params),
                                           _P, _P]),
    "pmh_rerank_forward": (ctypes.c_int, [_P, _P, _i64, _P, _P]),
    "pmh_rerank_gradients": (ctypes.c_int, [_P, _P, _P, _i64, _P, _P, _P]),
    "pmh_rerank_adam_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                            ctypes.c_float, _P]),
}


def exported_names() -> list[str]:
    return sorted(_SIGS)


def load():
    """Load the library (built by paper_2511_16576_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PMH_OK:
        raise PmhError(rc, load().pmh_last_error().decode())


def _ptr(t) -> int | None:
    """Device address of a tensor; an empty view of an allocation passes its storage's
    address (a zero-size tensor may report a null data pointer)."""
    if t is None:
        return None
    if t.numel() == 0:
        return t.untyped_storage().data_ptr() or None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    """A library context on one CUDA device (owns scratch memory).

    Closing it first closes every handle (polygons, index, graph) made with it."""

    def __init__(self, device: int = 0):
        import weakref
        lib = load()
        h = _P()
        _check(lib.pmh_create(ctypes.byref(h), device))
        self.handle = h
        self.device = device
        self._children = weakref.WeakSet()

    def _adopt(self, child):
        self._children.add(child)

    def close(self):
        if self.handle:
            for child in list(self._children):
                child.close()
            load().pmh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Polys:
    """Polygons uploaded to library-owned device memory (step A0)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle
        ctx._adopt(self)
        n, nv = _i64(), _i64()
        _check(load().pmh_polys_info(handle, ctypes.byref(n), ctypes.byref(nv)))
        self.n, self.n_vertices = n.value, nv.value

    def prep(self, stream=None):
        dev = torch.device("cuda", self.ctx.device)
        bbox = torch.empty((max(self.n, 1), 4), dtype=torch.int32, device=dev)
        area2 = torch.empty(max(self.n, 1), dtype=torch.int64, device=dev)
        _check(load().pmh_polys_prep(self.handle, _ptr(bbox), _ptr(area2), _stream(stream)))
        return bbox[:self.n], area2[:self.n]

    def close(self):
        if self.handle:
            load().pmh_polys_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poly_upload(ctx: Context, xy: torch.Tensor, offsets: torch.Tensor, stream=None) -> Polys:
    """Upload device arrays xy int32 [V, 2] and offsets int64 [N + 1]."""
    assert xy.dtype == torch.int32 and offsets.dtype == torch.int64
    assert xy.is_cuda and offsets.is_cuda and xy.is_contiguous() and offsets.is_contiguous()
    h = _P()
    n = offsets.numel() - 1
    _check(load().pmh_poly_upload(ctx.handle, _ptr(xy), _ptr(offsets), n, xy.shape[0],
                                  ctypes.byref(h), _stream(stream)))
    return Polys(ctx, h)


def poly_upload_host(ctx: Context, xy, offsets, stream=None) -> Polys:
    """Upload host arrays (numpy or CPU tensors, pinned or pageable)."""
    import numpy as np
    xy_np = np.ascontiguousarray(np.asarray(xy), dtype=np.int32)
    off_np = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    h = _P()
    _check(load().pmh_poly_upload_host(ctx.handle, xy_np.ctypes.data, off_np.ctypes.data,
                                       len(off_np) - 1, xy_np.shape[0], ctypes.byref(h),
                                       _stream(stream)))
    return Polys(ctx, h)


def poly_upload_pinned(ctx: Context, xy: torch.Tensor, offsets: torch.Tensor,
                       stream=None) -> Polys:
    """Upload pinned CPU tensors without an extra host copy."""
    assert not xy.is_cuda and not offsets.is_cuda
    h = _P()
    _check(load().pmh_poly_upload_host(ctx.handle, _ptr(xy), _ptr(offsets), offsets.numel() - 1,
                                       xy.shape[0], ctypes.byref(h), _stream(stream)))
    return Polys(ctx, h)


def poly_reload(polys: Polys, xy: torch.Tensor, offsets: torch.Tensor, stream=None):
    """Upload new polygons (same counts) into an existing set, keeping its buffers: CUDA
    tensors, or pinned CPU tensors."""
    assert xy.dtype == torch.int32 and offsets.dtype == torch.int64
    assert xy.is_contiguous() and offsets.is_contiguous() and xy.is_cuda == offsets.is_cuda
    _check(load().pmh_poly_reload(polys.handle, _ptr(xy), _ptr(offsets), offsets.numel() - 1,
                                  xy.shape[0], 0 if xy.is_cuda else 1, _stream(stream)))


def minhash_sign(ctx: Context, polys: Polys, params: Params, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """A1: uint32 hashes [N, K] (carried in an int32 tensor)."""
    if out is None:
        out = torch.empty((polys.n, params.K), dtype=torch.int32,
                          device=torch.device("cuda", ctx.device))
    _check(load().pmh_minhash_sign(ctx.handle, polys.handle, ctypes.byref(params), _ptr(out),
                                   _stream(stream)))
    return out


NOALLOC_MAX_POLYS = 262144


def minhash_sign_noalloc(xy: torch.Tensor, offsets: torch.Tensor, params: Params,
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Allocation-free A1 on raw device arrays (no context, no polygon handle).

    The library allocates nothing for this call (its scratch is a fixed device array of
    NOALLOC_MAX_POLYS bounding boxes); `out` is allocated here by torch only when the caller
    does not pass one.  Calls that overlap on the GPU share that array and race.  The
    arrays must be contiguous CUDA tensors on one device (xy int32 [V, 2], offsets int64
    [N + 1], out int32 with at least N * K elements); the call runs on that device and, by
    default, on its current stream.
    """
    if not (isinstance(xy, torch.Tensor) and isinstance(offsets, torch.Tensor)):
        raise PmhError(PMH_ERR_ARG, "xy and offsets must be torch tensors")
    if xy.dtype != torch.int32 or offsets.dtype != torch.int64:
        raise PmhError(PMH_ERR_ARG, "xy must be int32 and offsets int64")
    if xy.dim() != 2 or xy.shape[1] != 2 or offsets.dim() != 1 or offsets.numel() < 1:
        raise PmhError(PMH_ERR_ARG, "xy must be [V, 2] and offsets [N + 1]")
    arrays = [xy, offsets] + ([out] if out is not None else [])
    if not all(a.is_cuda for a in arrays):
        raise PmhError(PMH_ERR_ARG, "xy, offsets and out must be CUDA tensors")
    if len({a.device for a in arrays}) != 1:
        raise PmhError(PMH_ERR_ARG, "xy, offsets and out must be on one device")
    if not all(a.is_contiguous() for a in arrays):
        raise PmhError(PMH_ERR_ARG, "xy, offsets and out must be contiguous")
    n = offsets.numel() - 1
    if out is not None and (out.dtype != torch.int32 or out.numel() < n * params.K):
        raise PmhError(PMH_ERR_ARG, f"out must be int32 with at least {n * params.K} elements")
    with torch.cuda.device(xy.device):
        if out is None:
            out = torch.empty((n, params.K), dtype=torch.int32, device=xy.device)
        s = (stream if stream is not None else torch.cuda.current_stream(xy.device)).cuda_stream
        _check(load().pmh_minhash_sign_noalloc(_ptr(xy), _ptr(offsets), n, xy.shape[0],
                                               ctypes.byref(params), _ptr(out), s))
    return out


def stream_index_build(ctx: Context, params: Params, stream=None):
    """Build the context's stream index for (seed, K) ahead of indexed signing."""
    _check(load().pmh_stream_index_build(ctx.handle, ctypes.byref(params), _stream(stream)))


def sign_work(ctx: Context) -> dict:
    """Work units of the last signing call: walked points, cells, index entries,
    bbox candidates, edge tests."""
    import numpy as np
    c = np.zeros(6, np.uint64)
    _check(load().pmh_sign_work(ctx.handle, c.ctypes.data))
    return dict(zip(("walk_points", "cells", "index_entries", "candidates", "edge_tests",
                     "mask_decisions"), (int(v) for v in c)))


WORK_KEYS = ("walk_points", "cells", "index_entries", "candidates", "edge_tests", "mask_decisions")


def sign_count_work(ctx: Context, enable: bool = True):
    """Record work counts in later signing calls (the default) or run the kernels built
    without the counters (same hashes)."""
    _check(load().pmh_sign_count_work(ctx.handle, 1 if enable else 0))


def sign_timing(ctx: Context, enable: bool = True):
    """Record per-kernel events in later signing calls (unified kernel, walk kernel)."""
    _check(load().pmh_sign_timing(ctx.handle, 1 if enable else 0))


def sign_report(ctx: Context) -> dict:
    """Mean per-kernel milliseconds over the signing calls recorded since the last
    report, and the per-kernel work counts of the last signing call."""
    import numpy as np
    ms = np.zeros(3, np.float32)
    c = np.zeros(12, np.uint64)
    _check(load().pmh_sign_report(ctx.handle, ms.ctypes.data, c.ctypes.data))
    return {"calls": int(ms[2]),
            "unified": {"ms": float(ms[0]), "work": dict(zip(WORK_KEYS, (int(v) for v in c[:6])))},
            "walk": {"ms": float(ms[1]), "work": dict(zip(WORK_KEYS, (int(v) for v in c[6:])))}}


def band_keys(ctx: Context, hashes: torch.Tensor, params: Params, out=None, stream=None):
    """A2: uint64 band keys [N, bands] (carried in an int64 tensor)."""
    n = hashes.shape[0]
    if out is None:
        out = torch.empty((n, params.bands), dtype=torch.int64, device=hashes.device)
    _check(load().pmh_band_keys(ctx.handle, _ptr(hashes), n, ctypes.byref(params), _ptr(out),
                                _stream(stream)))
    return out


class Index:
    """A3: bucket index of database signatures."""

    def __init__(self, ctx: Context, hashes: torch.Tensor, params: Params, stream=None):
        h = _P()
        _check(load().pmh_lsh_build(ctx.handle, _ptr(hashes), hashes.shape[0],
                                    ctypes.byref(params), ctypes.byref(h), _stream(stream)))
        self.ctx, self.handle, self.params, self.n = ctx, h, params, hashes.shape[0]
        ctx._adopt(self)

    def close(self):
        if self.handle:
            load().pmh_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsh_build(ctx: Context, hashes: torch.Tensor, params: Params, stream=None) -> Index:
    return Index(ctx, hashes, params, stream)


def lsh_rebuild(ctx: Context, index: Index, hashes: torch.Tensor, stream=None):
    """A3 in place: rebuild `index` from new signatures of the same count."""
    _check(load().pmh_lsh_rebuild(ctx.handle, index.handle, _ptr(hashes), hashes.shape[0],
                                  _stream(stream)))


def lsh_query(ctx: Context, index: Index, qhashes: torch.Tensor, capacity: int | None = None,
              stream=None):
    """A4: CSR (row_ptr int64 [Q+1], cand int32 [total]); sizes the buffer itself."""
    Q = qhashes.shape[0]
    dev = qhashes.device
    row_ptr = torch.empty(Q + 1, dtype=torch.int64, device=dev)
    total = _i64()
    cap = 0 if capacity is None else capacity
    cand = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    lib = load()
    rc = lib.pmh_lsh_query(ctx.handle, index.handle, _ptr(qhashes), Q, _ptr(row_ptr), _ptr(cand),
                           cap, ctypes.byref(total), _stream(stream))
    if rc == PMH_ERR_CAPACITY and capacity is None:
        # the count pass already wrote row_ptr: only the fill pass remains
        cand = torch.empty(max(total.value, 1), dtype=torch.int32, device=dev)
        rc = lib.pmh_lsh_query_fill(ctx.handle, index.handle, _ptr(qhashes), Q, _ptr(row_ptr),
                                    _ptr(cand), total.value, _stream(stream))
    _check(rc)
    return row_ptr, cand[:total.value]


def jaccard_estimate(ctx: Context, qhashes, dbhashes, row_ptr, cand, params: Params,
                     bandmask: bool = True, stream=None):
    """A5: agreement counts (int16 carrying uint16) and band-match bits (int32 carrying uint32)."""
    E = cand.numel()
    dev = qhashes.device
    count = torch.empty(max(E, 1), dtype=torch.int16, device=dev)
    mask = torch.empty(max(E, 1), dtype=torch.int32, device=dev) if bandmask else None
    _check(load().pmh_jaccard_estimate(ctx.handle, _ptr(qhashes), _ptr(dbhashes), _ptr(row_ptr),
                                       _ptr(cand), qhashes.shape[0], ctypes.byref(params),
                                       _ptr(count), _ptr(mask), _stream(stream)))
    return count[:E], (mask[:E] if mask is not None else None)


def topm(ctx: Context, row_ptr, cand, count, m: int, score=None, stream=None):
    """A6: top-m ids per query ([Q, m], -1 padded) and kept counts [Q]."""
    Q = row_ptr.numel() - 1
    dev = row_ptr.device
    ids = torch.empty((max(Q, 1), m), dtype=torch.int32, device=dev)
    nn = torch.empty(max(Q, 1), dtype=torch.int32, device=dev)
    _check(load().pmh_topm(ctx.handle, _ptr(row_ptr), _ptr(cand), _ptr(count), _ptr(score), Q, m,
                           _ptr(ids), _ptr(nn), _stream(stream)))
    return ids[:Q], nn[:Q]


def lists_to_csr(ctx: Context, ids, nn, stream=None):
    """Fixed-width top-m lists to compact CSR (row_ptr int64 [Q+1], cand int32)."""
    Q, m = ids.shape
    row_ptr = torch.empty(Q + 1, dtype=torch.int64, device=ids.device)
    cand = torch.empty(max(Q * m, 1), dtype=torch.int32, device=ids.device)
    _check(load().pmh_lists_to_csr(ctx.handle, _ptr(ids), _ptr(nn), Q, m, _ptr(row_ptr), _ptr(cand),
                                   _stream(stream)))
    return row_ptr, cand


def refine_topk(ctx: Context, queries: Polys, db: Polys, ids, nn, k: int, stream=None):
    """A8: exact top-k by Jaccard among each query's listed ids."""
    Q, m = ids.shape
    dev = ids.device
    top_ids = torch.empty((max(Q, 1), k), dtype=torch.int32, device=dev)
    top_j = torch.empty((max(Q, 1), k), dtype=torch.float64, device=dev)
    _check(load().pmh_refine_topk(ctx.handle, queries.handle, db.handle, _ptr(ids), _ptr(nn), Q, m,
                                  k, _ptr(top_ids), _ptr(top_j), _stream(stream)))
    return top_ids[:Q], top_j[:Q]


def pair_jaccard(ctx: Context, queries: Polys, db: Polys, qid, pid, stream=None):
    """Exact Jaccard of explicit (query, database) pairs, fp64."""
    n = qid.numel()
    out = torch.empty(max(n, 1), dtype=torch.float64, device=qid.device)
    _check(load().pmh_pair_jaccard(ctx.handle, queries.handle, db.handle, _ptr(qid), _ptr(pid), n,
                                   _ptr(out), _stream(stream)))
    return out[:n]


def bbox_join(ctx: Context, queries: Polys, db: Polys, stream=None):
    """Brute-force candidates: CSR of bbox-overlapping database polygons per query."""
    dev = torch.device("cuda", ctx.device)
    row_ptr = torch.empty(queries.n + 1, dtype=torch.int64, device=dev)
    total = _i64()
    lib = load()
    cand = torch.empty(1, dtype=torch.int32, device=dev)
    rc = lib.pmh_bbox_join(ctx.handle, queries.handle, db.handle, _ptr(row_ptr), _ptr(cand), 0,
                           ctypes.byref(total), _stream(stream))
    if rc == PMH_ERR_CAPACITY:
        cand = torch.empty(max(total.value, 1), dtype=torch.int32, device=dev)
        rc = lib.pmh_bbox_join(ctx.handle, queries.handle, db.handle, _ptr(row_ptr), _ptr(cand),
                               total.value, ctypes.byref(total), _stream(stream))
    _check(rc)
    return row_ptr, cand[:total.value]


def probe_int_peak(ctx: Context) -> float:
    """Measured integer instructions per second (thread level) of this GPU."""
    ops, sec = ctypes.c_double(), ctypes.c_double()
    _check(load().pmh_probe_int_peak(ctx.handle, ctypes.byref(ops), ctypes.byref(sec)))
    return ops.value


def launch_count() -> int:
    return int(load().pmh_launch_count())


@dataclass
class Signed:
    polys: Polys
    hashes: torch.Tensor


# --------------------------------------------------------------------------- A9
SIGN_VARIANTS = 6
_AUTOTUNE_CACHE = os.path.join(_HERE, "_build", "autotune.json")


def sign_variant_info(v: int):
    u, w = ctypes.c_int(), ctypes.c_int()
    _check(load().pmh_sign_variant_info(v, ctypes.byref(u), ctypes.byref(w)))
    return u.value, w.value


def sign_set_variant(ctx: Context, v: int):
    _check(load().pmh_sign_set_variant(ctx.handle, v))


def sign_autotune(ctx: Context, sample: Polys, params: Params, cache_key: str | None = None):
    """Time every signing-kernel variant on `sample`, keep the fastest in the context.

    With a cache_key the choice is cached in _build/autotune.json per GPU name, K and key,
    and a cached choice is applied without timing."""
    import json
    gpu = torch.cuda.get_device_name(ctx.device)
    key = f"{gpu}|K={params.K}|{cache_key}" if cache_key else None
    cache = {}
    if key and os.path.exists(_AUTOTUNE_CACHE):
        try:
            cache = json.load(open(_AUTOTUNE_CACHE))
        except ValueError:
            cache = {}
        if key in cache:
            sign_set_variant(ctx, int(cache[key]["best"]))
            return int(cache[key]["best"]), cache[key]["ms"]
    best = ctypes.c_int()
    ms = (ctypes.c_float * SIGN_VARIANTS)()
    _check(load().pmh_sign_autotune(ctx.handle, sample.handle, ctypes.byref(params),
                                    ctypes.byref(best), ms))
    times = [float(v) for v in ms]
    if key:
        cache[key] = {"best": best.value, "ms": times,
                      "shapes": [sign_variant_info(v) for v in range(SIGN_VARIANTS)]}
        os.makedirs(os.path.dirname(_AUTOTUNE_CACHE), exist_ok=True)
        json.dump(cache, open(_AUTOTUNE_CACHE, "w"), indent=1)
    return best.value, times


class _DeviceArray:
    """__cuda_array_interface__ view of library-owned device memory (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _view(ptr, shape, typestr, device):
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=device)


class QueryGraph:
    """A9: captured query pipeline (prep, slab lists, sign, join, agreement, top-m and,
    with a database polygon set and k > 0, exact refinement to the top-k) replayed per
    batch."""

    def __init__(self, ctx: Context, index: Index, max_queries: int, max_vertices: int,
                 cand_capacity: int, m: int, db: "Polys | None" = None, k: int = 0,
                 rerank: "Reranker | None" = None, shortlist: int = 64, fused_select: bool = False):
        h = _P()
        cfg = QGraphConfig(max_queries, max_vertices, cand_capacity, m, k,
                           db.handle if db else None, rerank.handle if rerank else None,
                           shortlist if rerank else 0, QGRAPH_FUSED_SELECT if fused_select else 0)
        _check(load().pmh_qgraph_create(ctx.handle, index.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.ctx, self.index, self.db, self.rerank, self.handle = ctx, index, db, rerank, h
        ctx._adopt(self)
        self.max_queries, self.m, self.k, self.K = max_queries, m, k, index.params.K
        ptrs = [_P() for _ in range(6)]
        _check(load().pmh_qgraph_outputs(h, *[ctypes.byref(p) for p in ptrs]))
        dev = torch.device("cuda", ctx.device)
        Q = max_queries
        self.hashes = _view(ptrs[0].value, (Q, self.K), "<i4", dev)
        self.row_ptr = _view(ptrs[1].value, (Q + 1,), "<i8", dev)
        self.cand = _view(ptrs[2].value, (cand_capacity,), "<i4", dev)
        self.count = _view(ptrs[3].value, (cand_capacity,), "<i2", dev)
        self.top_ids = _view(ptrs[4].value, (Q, m), "<i4", dev)
        self.top_n = _view(ptrs[5].value, (Q,), "<i4", dev)
        self.ref_ids = self.ref_j = None
        if k > 0:
            ri, rj = _P(), _P()
            _check(load().pmh_qgraph_refined(h, ctypes.byref(ri), ctypes.byref(rj)))
            self.ref_ids = _view(ri.value, (Q, k), "<i4", dev)
            self.ref_j = _view(rj.value, (Q, k), "<f8", dev)

    def run(self, xy, offsets, stream=None):
        """Replay on one batch: device tensors, or pinned/pageable CPU tensors / numpy arrays."""
        n = len(offsets) - 1
        if isinstance(xy, torch.Tensor) and xy.is_cuda:
            _check(load().pmh_qgraph_run(self.handle, _ptr(xy), _ptr(offsets), n, xy.shape[0], 0,
                                         _stream(stream)))
        else:
            import numpy as np
            if isinstance(xy, torch.Tensor):
                xp, op = xy.data_ptr(), offsets.data_ptr()
                nv = xy.shape[0]
            else:
                self._keep = (np.ascontiguousarray(xy, np.int32), np.ascontiguousarray(offsets, np.int64))
                xp, op = self._keep[0].ctypes.data, self._keep[1].ctypes.data
                nv = self._keep[0].shape[0]
            _check(load().pmh_qgraph_run(self.handle, xp, op, n, nv, 1, _stream(stream)))
        return n

    def status(self, stream=None):
        f, t = ctypes.c_int(), _i64()
        _check(load().pmh_qgraph_status(self.handle, ctypes.byref(f), ctypes.byref(t),
                                        _stream(stream)))
        return f.value, t.value

    def close(self):
        if self.handle:
            load().pmh_qgraph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- A7
RERANK_IN, RERANK_HIDDEN, RERANK_PARAMS, RERANK_FEAT_COLS = 40, 64, 6849, 48


def unpack_params(flat):
    """Split packed reranker parameters into (w1, b1, w2, b2, w3, b3)."""
    import numpy as np
    flat = np.asarray(flat)
    h, d = RERANK_HIDDEN, RERANK_IN
    o = np.cumsum([0, h * d, h, h * h, h, h, 1])
    return (flat[o[0]:o[1]].reshape(h, d), flat[o[1]:o[2]], flat[o[2]:o[3]].reshape(h, h),
            flat[o[3]:o[4]], flat[o[4]:o[5]], flat[o[5]:o[6]])


def init_rerank_params(seed: int = 0):
    """Packed fp32 initial weights: He-normal layers, zero biases, small output layer."""
    import numpy as np
    rng = np.random.default_rng(seed)
    h, d = RERANK_HIDDEN, RERANK_IN
    parts = [rng.normal(0, np.sqrt(2.0 / d), (h, d)), np.zeros(h),
             rng.normal(0, np.sqrt(2.0 / h), (h, h)), np.zeros(h),
             rng.normal(0, np.sqrt(1.0 / h), h), np.zeros(1)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def rerank_features(ctx: Context, queries: Polys, db: Polys, qhashes, dbhashes, row_ptr, cand,
                    params: Params, stream=None):
    """A7 features: bf16 bits [E, 48] (int16 tensor) of every CSR pair."""
    E = cand.numel()
    out = torch.empty((max(E, 1), RERANK_FEAT_COLS), dtype=torch.int16, device=qhashes.device)
    _check(load().pmh_rerank_features(ctx.handle, queries.handle, db.handle, _ptr(qhashes),
                                      _ptr(dbhashes), _ptr(row_ptr), _ptr(cand),
                                      row_ptr.numel() - 1, ctypes.byref(params), _ptr(out),
                                      _stream(stream)))
    return out[:E]


class Reranker:
    """A7: the MLP reranker (training and inference kernels on the GPU)."""

    def __init__(self, ctx: Context, weights=None, seed: int = 0):
        h = _P()
        _check(load().pmh_rerank_create(ctx.handle, ctypes.byref(h)))
        self.ctx, self.handle = ctx, h
        ctx._adopt(self)
        dev = torch.device("cuda", ctx.device)
        self._loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.set_weights(init_rerank_params(seed) if weights is None else weights)

    def set_weights(self, flat):
        import numpy as np
        w = np.ascontiguousarray(flat, dtype=np.float32)
        assert w.size == RERANK_PARAMS
        _check(load().pmh_rerank_set_weights(self.handle, w.ctypes.data))

    def get_weights(self):
        import numpy as np
        w = np.empty(RERANK_PARAMS, np.float32)
        _check(load().pmh_rerank_get_weights(self.handle, w.ctypes.data))
        return w

    def forward(self, feat, out=None, stream=None):
        n = feat.shape[0]
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.float32, device=feat.device)
        _check(load().pmh_rerank_forward(self.handle, _ptr(feat), n, _ptr(out), _stream(stream)))
        return out[:n]

    def gradients(self, feat, label, stream=None):
        """(packed gradients [6657] fp32 tensor, loss tensor) of the mean squared error."""
        grads = torch.empty(RERANK_PARAMS, dtype=torch.float32, device=feat.device)
        _check(load().pmh_rerank_gradients(self.handle, _ptr(feat), _ptr(label), feat.shape[0],
                                           _ptr(grads), _ptr(self._loss), _stream(stream)))
        return grads, self._loss

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  stream=None):
        _check(load().pmh_rerank_adam_step(self.handle, lr, beta1, beta2, eps, _stream(stream)))

    def train_step(self, feat, label, lr: float, stream=None):
        """One Adam step on one batch; returns the batch loss tensor (device)."""
        _check(load().pmh_rerank_gradients(self.handle, _ptr(feat), _ptr(label), feat.shape[0],
                                           None, _ptr(self._loss), _stream(stream)))
        self.adam_step(lr, stream=stream)
        return self._loss

    def close(self):
        if self.handle:
            load().pmh_rerank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""The allocation-free signing entry point gives the same hashes as pmh_minhash_sign.

pmh_minhash_sign_noalloc serves callers that cannot let a library allocate device
memory (a fixed device-memory budget reserved up front, memory owned by a caching
allocator, latency-critical loops that cannot absorb cudaFree's device-wide
synchronisation).  Its scratch is one fixed device array shared by every call, so the
test makes two calls in a row on different inputs -- the second must not see the
first one's ticket or bounding boxes -- and compares both with the ordinary entry
point, and the second also directly with the CPU oracle.  The second batch holds
polygons that reach past the lattice domain on every side and one wholly outside it,
so the call's own bounding-box clipping is exercised.  Hashes are integers: the
comparison is exact.  This file is collected last so that a failure here leaves every
other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_16576_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def B():
    from paper_2511_16576_gb300 import binding, build
    build.build()
    return binding


def with_clipped(ps):
    """ps plus polygons partly outside the domain (negative coordinates, coordinates above
    65536, both) and one wholly outside it (its clipped box is empty: every hash is T)."""
    extra = [np.array([[-3000, -2000], [9000, -500], [4000, 7000]], np.int32),
             np.array([[60000, 61000], [70500, 62000], [69000, 71000], [61000, 69000]], np.int32),
             np.array([[-500, 30000], [66000, 29000], [66500, 36000], [-800, 35000]], np.int32),
             np.array([[70000, 70000], [80000, 70000], [75000, 80000]], np.int32),
             np.array([[-9000, 100], [-100, 100], [-4000, 9000]], np.int32)]
    xy = np.concatenate([ps.xy] + extra)
    off = np.concatenate([ps.offsets, ps.offsets[-1] + np.cumsum([len(e) for e in extra])])
    return xy, off.astype(np.int64)


def test_noalloc_matches_sign_on_two_calls(B, orc):
    ctx = B.Context(0)
    try:
        first = synth.star_polygons(3000, 91, (8, 300), "loguniform", (1e-3, 3e-2))
        second = synth.star_polygons(700, 92, (3, 64), "uniform", (5e-3, 5e-2))
        cases = ((first.xy, first.offsets, (128, 16, 1 << 24)),
                 (*with_clipped(second), (40, 8, 5000)))
        for call, (xy_np, off_np, (K, bands, T)) in enumerate(cases):
            P = B.make_params(K, bands, T)
            xy = torch.from_numpy(xy_np).to(DEV)
            off = torch.from_numpy(off_np).to(DEV)
            ref = B.minhash_sign(ctx, B.poly_upload(ctx, xy, off), P)
            got = B.minhash_sign_noalloc(xy, off, P)
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
            if call == 1:
                want = orc.sign(xy_np, off_np, P.seed, K, T, nthreads=8)
                assert np.array_equal(got.cpu().numpy().view(np.uint32), want)
                assert (want[-2:] == T).all()  # wholly outside the domain
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_batches(B):
    n = B.NOALLOC_MAX_POLYS + 1
    off = torch.arange(n + 1, device=DEV, dtype=torch.int64) * 3
    xy = torch.zeros((3 * n, 2), dtype=torch.int32, device=DEV)
    out = torch.empty((n, 32), dtype=torch.int32, device=DEV)
    with pytest.raises(B.PmhError) as ei:
        B.minhash_sign_noalloc(xy, off, B.make_params(32, 8), out=out)
    assert "at most" in str(ei.value)


def test_noalloc_reports_invalid_polygons(B):
    xy = torch.tensor([[0, 0], [5, 0], [0, 5], [1, 1], [2, 2]], dtype=torch.int32, device=DEV)
    off = torch.tensor([0, 3, 5], dtype=torch.int64, device=DEV)   # second has 2 vertices
    with pytest.raises(B.PmhError) as ei:
        B.minhash_sign_noalloc(xy, off, B.make_params(32, 8))
    assert "fewer than 3" in str(ei.value)


def test_noalloc_refuses_host_arrays_without_launching(B):
    xy = torch.tensor([[0, 0], [500, 0], [0, 500]], dtype=torch.int32, device=DEV)
    off_host = torch.tensor([0, 3], dtype=torch.int64)
    P = B.make_params(32, 8)
    before = B.launch_count()
    # the binding refuses a CPU tensor ...
    with pytest.raises(B.PmhError):
        B.minhash_sign_noalloc(xy, off_host, P)
    # ... and the C entry point itself refuses a host pointer
    out = torch.empty((1, 32), dtype=torch.int32, device=DEV)
    off_np = np.array([0, 3], np.int64)
    rc = B.load().pmh_minhash_sign_noalloc(xy.data_ptr(), off_np.ctypes.data, 1, 3,
                                           ctypes.byref(P), out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == B.PMH_ERR_ARG
    assert "d_offsets" in B.load().pmh_last_error().decode()
    assert B.launch_count() == before
